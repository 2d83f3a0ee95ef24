// Internal declarations shared by the translation units of libgvs.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gvs.h"

namespace gvs {

// Multiprocessor count of the current device (queried once per device).
int device_sm_count();

// Per-view FP32 coefficients of the address contract (see gvs.h).
struct ViewXform {
    float M[9];
    float b[3];
};

// ---- temporal refinement -------------------------------------------------
cudaError_t launch_refine(const uint32_t *rgba_t, const uint32_t *rgba_prev, const float *depth_t,
                          float *state, uint8_t *mask, int64_t n, int threshold, cudaStream_t st);

// ---- TSDF fusion -----------------------------------------------------------
// Byte layout of the fusion workspace ("map"): the packed (depth, weight)
// float2 per input pixel, then per-view depth bounds (min, max over valid
// depths; +inf/-inf where a tile has none) over 8x8, 32x32 and 128x128 pixel
// tiles and over the whole view.  Every section starts 256-byte aligned.
struct MapLayout {
    int K, W, H;
    int t3w, t3h, t5w, t5h, t7w, t7h;
    size_t off_dw, off_t3, off_t5, off_t7, off_g, total;
};

inline MapLayout map_layout(int K, int W, int H) {
    auto up = [](size_t n) { return (n + 255) / 256 * 256; };
    MapLayout m;
    m.K = K; m.W = W; m.H = H;
    m.t3w = (W + 7) >> 3;    m.t3h = (H + 7) >> 3;
    m.t5w = (W + 31) >> 5;   m.t5h = (H + 31) >> 5;
    m.t7w = (W + 127) >> 7;  m.t7h = (H + 127) >> 7;
    size_t o = 0;
    m.off_dw = o; o = up(o + (size_t)K * W * H * 8);
    m.off_t3 = o; o = up(o + (size_t)K * m.t3w * m.t3h * 8);
    m.off_t5 = o; o = up(o + (size_t)K * m.t5w * m.t5h * 8);
    m.off_t7 = o; o = up(o + (size_t)K * m.t7w * m.t7h * 8);
    m.off_g = o;  o = up(o + (size_t)K * 8);
    m.total = K > 0 ? o : 0;
    return m;
}

struct FuseArgs {
    const float2 *dw;          // [K][H][W] packed (depth or 0, weight)
    const float2 *t3, *t5, *t7, *tg;  // depth bounds per tile level and per view
    int t3w, t3h, t5w, t5h, t7w, t7h;
    int K, W, H;               // input views and their size
    int Wt, Ht;                // target size
    int D;
    float zn, dz, inv_mu;
    float behind;              // a sample is surely cut off where z > d_max + behind (= 1.0001 mu)
    int normalize;
    float *fused;
    int16_t *crossing;
    ViewXform xf[GVS_MAX_VIEWS];
};

cudaError_t launch_weight_map(const float *depth, void *map, int K, int W, int H, float mu, float wconst,
                              int window, cudaStream_t st);
cudaError_t launch_fuse(const FuseArgs &a, cudaStream_t st);

// ---- forward splat ---------------------------------------------------------
struct SplatView {
    ViewXform xf;
    float f_ratio;
};

struct SplatArgs {
    const float *depth;        // [K][H][W]
    const uint32_t *rgba;      // [K][H][W]
    int W, H, Wt, Ht;
    int footprint;
    float max_hw, mu_guide;
    const float *fused;        // [Ht][Wt] or null
    int32_t *winner;
    uint32_t *warped_rgba;
    float *warped_depth;
    uint8_t *alpha;
    uint8_t *guided;
    unsigned long long *keys;  // [slots][Ht][Wt]
    int slots;
    SplatView v[GVS_MAX_VIEWS];
};

cudaError_t launch_splat(const SplatArgs &a, int K, cudaStream_t st);

}  // namespace gvs
