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
// depth_dtype: GVS_F32 or GVS_F16 (depth_t and state share it)
cudaError_t launch_refine(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state,
                          uint8_t *mask, int64_t n, int threshold, int depth_dtype, cudaStream_t st);

// ws: 2 * K * ceil(W/4) * ceil(H/4) floats
cudaError_t launch_refine_soft(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state,
                               float *mask, int K, int W, int H, float beta, float lambda_t, int depth_dtype,
                               float *ws, cudaStream_t st);

// ---- TSDF fusion -----------------------------------------------------------
// Byte layout of the fusion workspace ("map"): the packed (depth, weight)
// float2 per input pixel, then per-view depth bounds.  For each tile level l
// in {4, 5, 6, 7} (tiles of 2^l x 2^l pixels) T_l holds the bounds of each
// tile and O_l the bounds of the 2x2 block of tiles anchored at it, so that
// any pixel box spanning at most two tiles per axis at level l is covered by
// one O_l entry.  G holds the bounds of the whole view.  Sections are 256-byte
// aligned.  A bound (DepthBound) is the smallest and largest valid depth of
// its pixels (+inf / -inf where there is none) and a 64-bit mask of occupied
// depth bins.  The bins are those of the FP32 bit pattern: bin(d) = bits(d)
// >> 18 (exponent and the 5 leading mantissa bits: 32 bins per octave, 1.6 to
// 3.1 % of the depth wide), monotone in d for d >= 0 and exact.  Bit b of a
// bound's mask is set when some valid depth d of its pixels has
// bin(d) - bin(lo) = b, or >= 63 for b = 63.  A coarser bound takes its
// children's masks shifted by the difference of their bin(lo) (whatever moves
// past bit 63 lands on bit 63), so a clear bit proves that no depth of the
// pixels lies in that bin.  G's mask is all ones (it is never consulted).
struct __align__(16) DepthBound {
    float lo, hi;
    unsigned mlo, mhi;  // bins 0..31, 32..63
};
constexpr int kBoundLevels = 4;    // levels 4, 5, 6, 7
constexpr int kBoundShift0 = 4;    // finest tile: 16 x 16 pixels
constexpr int kDepthBins = 64;

struct MapLayout {
    int K, W, H;
    int tw[kBoundLevels], th[kBoundLevels];  // tiles per row / column at levels 4..7
    size_t off_dw, off_T[kBoundLevels], off_O[kBoundLevels], off_g, total;
};

inline MapLayout map_layout(int K, int W, int H) {
    auto up = [](size_t n) { return (n + 255) / 256 * 256; };
    MapLayout m;
    m.K = K; m.W = W; m.H = H;
    size_t o = 0;
    m.off_dw = o; o = up(o + (size_t)K * W * H * 8);
    for (int l = 0; l < kBoundLevels; ++l) {
        const int sh = kBoundShift0 + l;
        m.tw[l] = (W + (1 << sh) - 1) >> sh;
        m.th[l] = (H + (1 << sh) - 1) >> sh;
        m.off_T[l] = o; o = up(o + (size_t)K * m.tw[l] * m.th[l] * sizeof(DepthBound));
        m.off_O[l] = o; o = up(o + (size_t)K * m.tw[l] * m.th[l] * sizeof(DepthBound));
    }
    m.off_g = o; o = up(o + (size_t)K * sizeof(DepthBound));
    m.total = K > 0 ? o : 0;
    return m;
}

#ifdef __CUDACC__
// Depth bin of a value d >= 0 (see DepthBound); the same integer arithmetic in
// the map build and in the slab test.
__device__ __forceinline__ int depth_bin(float d) { return (int)(__float_as_uint(d) >> 18); }
#endif

struct FuseArgs {
    const void *dw;            // [K][H][W] packed (depth or 0, weight): float2 or half2 (map_dtype)
    int map_dtype;
    const DepthBound *ob[kBoundLevels];  // O_l overlapping 2x2-tile bounds, levels 4..7: [K][th][tw]
    const DepthBound *tg;                // whole-view bounds [K]
    int tw[kBoundLevels], th[kBoundLevels];
    int K, W, H;               // input views and their size
    int Wt, Ht;                // target size
    int D;
    float zn, dz, inv_mu;
    float behind;              // a sample is surely cut off where z > d_max + behind (= 1.0001 mu)
    int normalize;
    int variant;               // bundle shape / slab-test lengths (same result, different speed)
    // temporal term (Supplement A.2): per target pixel the previous output depth and its
    // weight, added as one more input at the ray's own pixel; null when absent
    const float *tmp_depth;
    const float *tmp_weight;
    float *wview;              // out: the input views' weight at the crossing (or null)
    float *fused;
    int16_t *crossing;
    ViewXform xf[GVS_MAX_VIEWS];
    const char *vb[GVS_MAX_VIEWS];  // view k's map plane: dw + k W H map elements
};

// exact: correctly rounded weight (float2 maps only; see weight_map_kernel)
cudaError_t launch_weight_map(const void *depth, int depth_dtype, void *map, int map_dtype, int K, int W, int H,
                              float mu, float wconst, int window, cudaStream_t st, bool exact = false);
cudaError_t launch_fuse(const FuseArgs &a, cudaStream_t st);

// One (frame, target) item of a batched fusion: its arguments and the index
// of its first bundle in the batch's bundle numbering.
struct BatchItem {
    FuseArgs args;
    int bundle_begin;
};
int bundle_count(int Wt, int Ht, int K, int variant);
cudaError_t launch_fuse_batch(const BatchItem *items, int n_items, int total, unsigned *counter, int K, int map_dtype,
                              int variant, cudaStream_t st);
// acc: [K][H][W] float2 scratch; grad_depths written (not accumulated)
cudaError_t launch_fuse_backward(const FuseArgs &a, const void *depth, int depth_dtype, const int16_t *crossing,
                                 const float *grad_fused, float *grad_depths, float2 *acc, float mu, float wconst,
                                 int window, cudaStream_t st);

// ---- forward splat ---------------------------------------------------------
struct SplatView {
    ViewXform xf;
    float f_ratio;
};

struct SplatArgs {
    const void *depth;         // [K][H][W] of depth_dtype
    int depth_dtype;
    const uint32_t *rgba;      // [K][H][W]
    int W, H, Wt, Ht;
    int footprint;
    int guide_reject;          // drop candidates with z < fused - mu_guide before the depth test
    float max_hw, mu_guide;
    const float *fused;        // [Ht][Wt] or null
    int32_t *winner;
    uint32_t *warped_rgba;
    float *warped_depth;
    uint8_t *alpha;
    uint8_t *guided;
    unsigned long long *keys;  // [slots][Ht][Wt]
    int slots;
    // differentiable colour splat (soft): colour [K][H][W][4] of color_dtype (F32 or BF16)
    const void *color;
    int color_dtype;
    float mu_band;
    float4 *acc;               // [slots][Ht][Wt] running (sum g c, sum g)
    float4 *out_color;         // [K][Ht][Wt] RGBA (A = 0)
    float *wsum;               // [K][Ht][Wt] sum g
    const float4 *grad_color;  // backward inputs [K][Ht][Wt]
    const float4 *grad_pixel;  // or one per target pixel for every view: (d/d colour rgb, d/d warped depth)
    const float *grad_depth;   // [K][Ht][Wt] or null
    float *grad_in_depth;      // backward outputs [K][H][W]
    float4 *grad_in_color;     // [K][H][W]
    SplatView v[GVS_MAX_VIEWS];
};

cudaError_t launch_splat(const SplatArgs &a, int K, cudaStream_t st);
// ---- the uniform-blend training loss ---------------------------------------
struct BlendLossLayout {
    int nblocks;
    size_t off_code, off_partial, off_scale, total;
};
BlendLossLayout blend_loss_layout(int64_t HWt);
// loss: device double[3] = {L, L1, L_Depth}; grad_pixel / grad_fused may be null
cudaError_t launch_blend_loss(int K, int64_t HWt, const float4 *color, const uint8_t *alpha, const float *wdepth,
                              const float *fused, const float *gt, float w_l1, float w_depth, double *loss,
                              float4 *grad_pixel, float *grad_fused, char *ws, cudaStream_t st);
// The gradient of the loss the last launch_blend_loss on ws computed, times *grad_loss
// (device float; null for 1).  grad_pixel / grad_fused may be null.
cudaError_t launch_blend_loss_grad(int64_t HWt, const char *ws, const float *grad_loss, float4 *grad_pixel,
                                   float *grad_fused, cudaStream_t st);

// Bulk copies whose wait gave up since the last call (read and cleared).
unsigned async_timeouts_take();
cudaError_t launch_soft_splat(const SplatArgs &a, int K, cudaStream_t st);
cudaError_t launch_temporal_weight(const void *masks, int mask_dtype, const int32_t *winner, int K, int64_t HW,
                                   int64_t HWt, const float *w_tmp_prev, const float *w_view_prev, float beta_t,
                                   float eta, float *w_tmp, float *target_mask, cudaStream_t st);
cudaError_t launch_guided_mask(const float *warped_depth, const uint8_t *alpha, const float *fused, int K,
                               int64_t HWt, float mu_guide, uint8_t *guided, cudaStream_t st);
cudaError_t launch_soft_splat_backward(const SplatArgs &a, int K, cudaStream_t st);

}  // namespace gvs
