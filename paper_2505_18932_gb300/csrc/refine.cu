// Temporal depth refinement, Sec. 3.2 Eq. 1-2 with a hard difference mask.
//
// HBM-bound streaming kernel: per pixel it reads two RGBA8 words, the new
// depth and the previous filtered depth (16 B with FP32 depth, 12 B with FP16)
// and writes the filtered depth and the mask byte (5 B or 3 B).  Four pixels
// per thread so that every access is a vector; a scalar tail covers n % 4.
// Depths are moved as raw bits, so the copy is exact in either format.
#include "gvs_internal.cuh"

namespace gvs {
namespace {

// 1 where any of R, G, B differs by more than T (alpha byte ignored).
__device__ __forceinline__ uint32_t changed(uint32_t a, uint32_t b, uint32_t T4) {
    uint32_t gt = __vcmpgtu4(__vabsdiffu4(a, b), T4);  // 0xff per byte where |a-b| > T
    return (gt & 0x00ffffffu) != 0u;
}

// Bit-exact select of four depths: FP32 (four words) or FP16 (four half-words in a uint2).
__device__ __forceinline__ uint4 select4(uint4 d, uint4 s, uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
    return make_uint4(m0 ? d.x : s.x, m1 ? d.y : s.y, m2 ? d.z : s.z, m3 ? d.w : s.w);
}
__device__ __forceinline__ uint2 select4(uint2 d, uint2 s, uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
    const uint32_t lo = (m0 ? 0x0000ffffu : 0u) | (m1 ? 0xffff0000u : 0u);
    const uint32_t hi = (m2 ? 0x0000ffffu : 0u) | (m3 ? 0xffff0000u : 0u);
    return make_uint2((d.x & lo) | (s.x & ~lo), (d.y & hi) | (s.y & ~hi));
}

// V: uint4 (four FP32 depths) or uint2 (four FP16 depths), moved as raw bits.
template <typename V>
__global__ void __launch_bounds__(256) refine_vec4(const uint4 *__restrict__ rgba_t, const uint4 *__restrict__ rgba_prev,
                                                   const V *__restrict__ depth_t, V *__restrict__ state,
                                                   uint32_t *__restrict__ mask, int64_t n4, uint32_t T4) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const V d = __ldcs(&depth_t[q]);
        V out;
        uint32_t m;
        if (rgba_prev) {
            const uint4 a = __ldcs(&rgba_t[q]);
            const uint4 b = __ldcs(&rgba_prev[q]);
            const uint32_t m0 = changed(a.x, b.x, T4), m1 = changed(a.y, b.y, T4);
            const uint32_t m2 = changed(a.z, b.z, T4), m3 = changed(a.w, b.w, T4);
            out = select4(d, state[q], m0, m1, m2, m3);
            m = m0 | (m1 << 8) | (m2 << 16) | (m3 << 24);
        } else {
            out = d;
            m = 0x01010101u;
        }
        state[q] = out;
        if (mask) mask[q] = m;
    }
}

// T: uint32_t (FP32 bits) or uint16_t (FP16 bits).
template <typename T>
__global__ void refine_tail(const uint32_t *__restrict__ rgba_t, const uint32_t *__restrict__ rgba_prev,
                            const T *__restrict__ depth_t, T *__restrict__ state, uint8_t *__restrict__ mask,
                            int64_t begin, int64_t n, uint32_t T4) {
    const int64_t p = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t m = rgba_prev ? changed(rgba_t[p], rgba_prev[p], T4) : 1u;
    if (m) state[p] = depth_t[p];
    if (mask) mask[p] = (uint8_t)m;
}

template <typename V, typename T>
void launch_typed(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state, uint8_t *mask,
                  int64_t n, uint32_t T4, cudaStream_t st) {
    const int64_t n4 = n / 4;
    if (n4 > 0) {
        int64_t blocks = (n4 + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (blocks > cap) blocks = cap;
        refine_vec4<V><<<(unsigned)blocks, 256, 0, st>>>(
            reinterpret_cast<const uint4 *>(rgba_t), reinterpret_cast<const uint4 *>(rgba_prev),
            reinterpret_cast<const V *>(depth_t), reinterpret_cast<V *>(state), reinterpret_cast<uint32_t *>(mask), n4,
            T4);
    }
    if (n - 4 * n4 > 0)
        refine_tail<T><<<1, 32, 0, st>>>(rgba_t, rgba_prev, reinterpret_cast<const T *>(depth_t),
                                         reinterpret_cast<T *>(state), mask, 4 * n4, n, T4);
}

}  // namespace

cudaError_t launch_refine(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state,
                          uint8_t *mask, int64_t n, int threshold, int depth_dtype, cudaStream_t st) {
    const uint32_t T = (uint32_t)(threshold < 0 ? 0 : (threshold > 255 ? 255 : threshold));
    const uint32_t T4 = T * 0x01010101u;
    if (depth_dtype == GVS_F16)
        launch_typed<uint2, uint16_t>(rgba_t, rgba_prev, depth_t, state, mask, n, T4, st);
    else
        launch_typed<uint4, uint32_t>(rgba_t, rgba_prev, depth_t, state, mask, n, T4, st);
    return cudaGetLastError();
}

}  // namespace gvs
