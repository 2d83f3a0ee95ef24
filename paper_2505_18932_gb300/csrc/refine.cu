// Temporal depth refinement, Sec. 3.2 Eq. 1-2 with a hard difference mask.
//
// HBM-bound streaming kernel: per pixel it reads two RGBA8 words, the new
// depth and the previous filtered depth (16 B with FP32 depth, 12 B with FP16)
// and writes the filtered depth and the mask byte (5 B or 3 B).  Four pixels
// per thread so that every access is a vector; a scalar tail covers n % 4.
// Depths are moved as raw bits, so the copy is exact in either format.
#include <cuda_fp16.h>

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

// ---------------------------------------------------------------------------
// The paper's soft difference mask (Sec. 3.2, Eq. 1 and Eq. 2):
//   M = min(|I^t - I^{t-1}| / lambda_t + beta, 1) at quarter resolution,
//   3x3 max-pool, bilinear upsample,  D' = M D + (1 - M) D'_prev.
// Three small passes: quarter cells (4x4 block means of the per-pixel largest
// channel difference), the pooled quarter grid, then the full-resolution
// upsample and blend.  Quarter grids live in the workspace.  Each pass runs on
// blocks of 32 x 8 cells or pixels with the view in blockIdx.z (no index division).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) soft_quarter(const uint32_t *__restrict__ rgba_t,
                                                    const uint32_t *__restrict__ rgba_prev, float *__restrict__ mq,
                                                    int W, int H, int Wq, int Hq, int K, float inv_lambda,
                                                    float beta) {
    const int qx = blockIdx.x * 32 + threadIdx.x, qy = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (qx >= Wq || qy >= Hq) return;
    const size_t q = ((size_t)k * Hq + qy) * Wq + qx;
    const size_t off = (size_t)k * W * H;
    float sum = 0.0f;
    int cnt = 0;
    for (int y = 4 * qy; y < min(4 * qy + 4, H); ++y)
        for (int x = 4 * qx; x < min(4 * qx + 4, W); ++x) {
            const size_t p = off + (size_t)y * W + x;
            const uint32_t d = __vabsdiffu4(__ldg(&rgba_t[p]), __ldg(&rgba_prev[p]));
            const uint32_t m = max(max(d & 0xffu, (d >> 8) & 0xffu), (d >> 16) & 0xffu);
            sum += (float)m;
            ++cnt;
        }
    const float mean = sum / (255.0f * (float)cnt);
    mq[q] = fminf(fmaf(mean, inv_lambda, beta), 1.0f);
}

__global__ void __launch_bounds__(256) soft_pool(const float *__restrict__ mq, float *__restrict__ pq, int Wq,
                                                 int Hq, int K) {
    const int qx = blockIdx.x * 32 + threadIdx.x, qy = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (qx >= Wq || qy >= Hq) return;
    const size_t q = ((size_t)k * Hq + qy) * Wq + qx;
    const float *m = mq + (size_t)k * Wq * Hq;
    float best = -1.0f;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int yy = min(max(qy + dy, 0), Hq - 1), xx = min(max(qx + dx, 0), Wq - 1);
            best = fmaxf(best, m[yy * Wq + xx]);
        }
    pq[q] = best;
}

__device__ __forceinline__ float ld_depth(const float *p) { return *p; }
__device__ __forceinline__ float ld_depth(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st_depth(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_depth(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ bool valid_d(float d) { return isfinite(d) && d > 0.0f; }

// SB_V consecutive pixels of a row per thread: they share the row's vertical
// interpolation terms and keep more loads in flight; each pixel's arithmetic is
// the single-pixel form, in the same order.
constexpr int SB_V = 4;

template <typename T>
__global__ void __launch_bounds__(256) soft_blend(const float *__restrict__ pq, const T *__restrict__ depth_t,
                                                  T *__restrict__ state, float *__restrict__ mask, int W, int H,
                                                  int Wq, int Hq, int K) {
    const int xs = (blockIdx.x * 32 + threadIdx.x) * SB_V, y = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (xs >= W || y >= H) return;
    const float *m = pq + (size_t)k * Wq * Hq;
    const float sy = fminf(fmaxf((y + 0.5f) * 0.25f - 0.5f, 0.0f), (float)(Hq - 1));
    const int y0 = (int)sy;
    const int y1 = min(y0 + 1, Hq - 1);
    const float fy = sy - (float)y0;
    const float *m0 = m + y0 * Wq, *m1 = m + y1 * Wq;
    const size_t row = ((size_t)k * H + y) * W;
#pragma unroll
    for (int e = 0; e < SB_V; ++e) {
        const int x = xs + e;
        if (x >= W) break;
        const size_t p = row + x;
        const float sx = fminf(fmaxf((x + 0.5f) * 0.25f - 0.5f, 0.0f), (float)(Wq - 1));
        const int x0 = (int)sx;
        const int x1 = min(x0 + 1, Wq - 1);
        const float fx = sx - (float)x0;
        const float M = (1.0f - fy) * ((1.0f - fx) * m0[x0] + fx * m0[x1]) + fy * ((1.0f - fx) * m1[x0] + fx * m1[x1]);
        if (mask) mask[p] = M;
        const float dn = ld_depth(&depth_t[p]), dp = ld_depth(&state[p]);
        float out;
        if (!valid_d(dp)) out = dn;
        else if (!valid_d(dn)) out = dp;
        else out = fmaf(M, dn - dp, dp);  // M dn + (1 - M) dp
        st_depth(&state[p], out);
    }
}

template <typename T>
cudaError_t launch_soft_typed(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state,
                              float *mask, int K, int W, int H, float beta, float lambda_t, float *ws,
                              cudaStream_t st) {
    const int Wq = (W + 3) / 4, Hq = (H + 3) / 4;
    const int64_t nq = (int64_t)K * Wq * Hq, n = (int64_t)K * W * H;
    float *mq = ws, *pq = ws + nq;
    (void)n;
    const dim3 block(32, 8), gq((Wq + 31) / 32, (Hq + 7) / 8, K), gp((W + 32 * SB_V - 1) / (32 * SB_V), (H + 7) / 8, K);
    soft_quarter<<<gq, block, 0, st>>>(rgba_t, rgba_prev, mq, W, H, Wq, Hq, K, 1.0f / lambda_t, beta);
    soft_pool<<<gq, block, 0, st>>>(mq, pq, Wq, Hq, K);
    soft_blend<T><<<gp, block, 0, st>>>(pq, reinterpret_cast<const T *>(depth_t), reinterpret_cast<T *>(state), mask,
                                        W, H, Wq, Hq, K);
    return cudaGetLastError();
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

cudaError_t launch_refine_soft(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t, void *state,
                               float *mask, int K, int W, int H, float beta, float lambda_t, int depth_dtype,
                               float *ws, cudaStream_t st) {
    return depth_dtype == GVS_F16
               ? launch_soft_typed<__half>(rgba_t, rgba_prev, depth_t, state, mask, K, W, H, beta, lambda_t, ws, st)
               : launch_soft_typed<float>(rgba_t, rgba_prev, depth_t, state, mask, K, W, H, beta, lambda_t, ws, st);
}

}  // namespace gvs
