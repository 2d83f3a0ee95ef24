// Temporal depth refinement, Sec. 3.2 Eq. 1-2 with a hard difference mask.
//
// HBM-bound streaming kernel: per pixel it reads two RGBA8 words, the new
// depth and the previous filtered depth (16 B) and writes the filtered depth
// and the mask byte (5 B).  Four pixels per thread so that every access is a
// 16-byte vector (the mask a 4-byte word); a scalar tail covers n % 4.
#include "gvs_internal.cuh"

namespace gvs {
namespace {

// 1 where any of R, G, B differs by more than T (alpha byte ignored).
__device__ __forceinline__ uint32_t changed(uint32_t a, uint32_t b, uint32_t T4) {
    uint32_t gt = __vcmpgtu4(__vabsdiffu4(a, b), T4);  // 0xff per byte where |a-b| > T
    return (gt & 0x00ffffffu) != 0u;
}

__global__ void __launch_bounds__(256) refine_vec4(const uint4 *__restrict__ rgba_t,
                                                   const uint4 *__restrict__ rgba_prev,
                                                   const float4 *__restrict__ depth_t,
                                                   float4 *__restrict__ state, uint32_t *__restrict__ mask,
                                                   int64_t n4, uint32_t T4) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const float4 d = __ldcs(&depth_t[q]);
        float4 out;
        uint32_t m;
        if (rgba_prev) {
            const uint4 a = __ldcs(&rgba_t[q]);
            const uint4 b = __ldcs(&rgba_prev[q]);
            const float4 s = state[q];
            const uint32_t m0 = changed(a.x, b.x, T4), m1 = changed(a.y, b.y, T4);
            const uint32_t m2 = changed(a.z, b.z, T4), m3 = changed(a.w, b.w, T4);
            out.x = m0 ? d.x : s.x;
            out.y = m1 ? d.y : s.y;
            out.z = m2 ? d.z : s.z;
            out.w = m3 ? d.w : s.w;
            m = m0 | (m1 << 8) | (m2 << 16) | (m3 << 24);
        } else {
            out = d;
            m = 0x01010101u;
        }
        state[q] = out;
        if (mask) mask[q] = m;
    }
}

__global__ void refine_tail(const uint32_t *__restrict__ rgba_t, const uint32_t *__restrict__ rgba_prev,
                            const float *__restrict__ depth_t, float *__restrict__ state,
                            uint8_t *__restrict__ mask, int64_t begin, int64_t n, uint32_t T4) {
    const int64_t p = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t m = rgba_prev ? changed(rgba_t[p], rgba_prev[p], T4) : 1u;
    if (m) state[p] = depth_t[p];
    if (mask) mask[p] = (uint8_t)m;
}

}  // namespace

cudaError_t launch_refine(const uint32_t *rgba_t, const uint32_t *rgba_prev, const float *depth_t, float *state,
                          uint8_t *mask, int64_t n, int threshold, cudaStream_t st) {
    const uint32_t T = (uint32_t)(threshold < 0 ? 0 : (threshold > 255 ? 255 : threshold));
    const uint32_t T4 = T * 0x01010101u;
    const int64_t n4 = n / 4;
    if (n4 > 0) {
        int64_t blocks = (n4 + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (blocks > cap) blocks = cap;
        refine_vec4<<<(unsigned)blocks, 256, 0, st>>>(
            reinterpret_cast<const uint4 *>(rgba_t), reinterpret_cast<const uint4 *>(rgba_prev),
            reinterpret_cast<const float4 *>(depth_t), reinterpret_cast<float4 *>(state),
            reinterpret_cast<uint32_t *>(mask), n4, T4);
    }
    const int64_t tail = n - 4 * n4;
    if (tail > 0) refine_tail<<<1, 32, 0, st>>>(rgba_t, rgba_prev, depth_t, state, mask, 4 * n4, n, T4);
    return cudaGetLastError();
}

}  // namespace gvs
