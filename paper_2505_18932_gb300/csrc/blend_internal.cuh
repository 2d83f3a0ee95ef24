// Blending-network input and blend (Sec. 3.3): arguments and launch entries
// shared by blend.cu and the C ABI.
#pragma once

#include "gvs_internal.cuh"

namespace gvs {

struct BlendArgs {
    int K, Wt, Ht;
    const uint32_t *rgba;      // [K][Ht][Wt] warped colour (RGBA8)
    const float *wdepth;       // [K][Ht][Wt] warped depth
    const uint8_t *alpha;      // [K][Ht][Wt]
    const float *fused;        // [Ht][Wt] TSDF depth
    float fx, fy, cx, cy;      // target intrinsics, rounded to FP32
    float ck[GVS_MAX_VIEWS][3];  // view centres in the target camera frame
    float dist[GVS_MAX_VIEWS];   // |c_k - c_t|
    float axis[GVS_MAX_VIEWS];   // optical-axis dot products z_k . z_t
};

cudaError_t launch_blend_features(const BlendArgs &a, int out_dtype, void *out, cudaStream_t st);
int blend_blocks(int Wt, int Ht);
cudaError_t launch_blend(const BlendArgs &a, int weight_dtype, const void *w, const void *w_bg, const void *i_bg,
                         float *image, double *l_depth, double *partial, cudaStream_t st);

}  // namespace gvs
