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
struct FuseArgs {
    const float2 *dw;          // [K][H][W] packed (depth or 0, weight)
    int K, W, H;               // input views and their size
    int Wt, Ht;                // target size
    int D;
    float zn, dz, inv_mu;
    int normalize;
    float *fused;
    int16_t *crossing;
    ViewXform xf[GVS_MAX_VIEWS];
};

cudaError_t launch_weight_map(const float *depth, float2 *dw, int K, int W, int H, float mu, float wconst,
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
