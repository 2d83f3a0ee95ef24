// The training loss of Sec. 3.3 on the uniform blend of the views (Eq. 4 with
// every w_k = 1, the denominator read as the sum over the views) and its
// gradient, for the differentiable splat's outputs:
//   A(p) = sum_k a_k(p),  B(p) = sum_k a_k I_k(p) / A(p)      (n pixels with A > 0)
//   L1 = sum_{A>0} sum_rgb |B - GT| / (3 n)
//   Dbar(p) = sum_k a_k D_k(p) / A(p),  v(p) = [A > 0 and F(p) > 0]
//   L_Depth = sum_p v |F - Dbar| / (K Ht Wt)
//   L = w_l1 L1 + w_depth L_Depth
// Three passes: per pixel the blend, the signs the gradient needs (packed in one
// 32-bit code) and per-block partial sums; one block adding the partials in a
// fixed order (so the loss is deterministic) and fixing the two scales; per
// pixel the gradient, scaled by the upstream gradient of L when one is given
// (read on the device, so a backward pass needs no host round trip).  Every
// view k with a_k = 1 at p receives the same d L / d I_k = g_rgb(p) and
// d L / d D_k = g_d(p), so they are written once per pixel (float4: g_rgb,
// g_d) instead of once per view; uncovered pixels get 0.
#include <math.h>

#include "gvs_internal.cuh"

namespace gvs {
namespace {

constexpr int BL_THREADS = 256;
// the pass's grid: 1216 blocks (2 waves of 4 resident blocks on 152 SMs) or one per
// 256 pixels when fewer
constexpr int kPassBlocks = 1216;
inline int pass_blocks(int64_t HWt) {
    const int64_t b = (HWt + BL_THREADS - 1) / BL_THREADS;
    return (int)(b < kPassBlocks ? b : kPassBlocks);
}

// code bits: 0-5 A (<= 32 views), 6-11 the signs of B - GT (2 bits per channel:
// 1 positive, 2 negative), 12-13 the sign of F - Dbar, 14 covered, 15 v.
__device__ __forceinline__ unsigned sign2(float x) { return x > 0.0f ? 1u : (x < 0.0f ? 2u : 0u); }
__device__ __forceinline__ float unsign2(unsigned s) { return s == 1u ? 1.0f : (s == 2u ? -1.0f : 0.0f); }

struct Partial {
    double l1, ld;
    unsigned long long n;
};

// A fixed grid (pass_blocks(HWt), a function of the size only) strides over the
// pixels, so there are few partials and the order of every sum is fixed.  Per
// pixel, per thread (a few pixels) and within a warp in FP32: the terms are
// non-negative, so each such sum is within (terms + 5) 2^-24 of its value
// relative to itself; FP64 from the warps' sums on.  FP64 arithmetic per pixel
// would run at a small fraction of the FP32 rate.
__global__ void __launch_bounds__(BL_THREADS, 4) blend_loss_pass(int K, int64_t HWt, const float4 *__restrict__ color,
                                                              const uint8_t *__restrict__ alpha,
                                                              const float *__restrict__ wdepth,
                                                              const float *__restrict__ fused,
                                                              const float *__restrict__ gt, unsigned *__restrict__ code,
                                                              Partial *__restrict__ partial) {
    __shared__ float s_l1[BL_THREADS / 32], s_ld[BL_THREADS / 32];
    __shared__ unsigned s_n[BL_THREADS / 32];
    float l1 = 0.0f, ld = 0.0f;
    unsigned n = 0;
    for (int64_t p = (int64_t)blockIdx.x * BL_THREADS + threadIdx.x; p < HWt; p += (int64_t)gridDim.x * BL_THREADS) {
        // B - GT = sum_k a_k (I_k - GT) / A and F - Dbar = sum_k a_k (F - D_k) / A: summing the
        // differences keeps a tie exact (each difference of equal values is 0, and a
        // difference of nearby values is exact), so the sign the gradient carries is the
        // exact sign of B - GT and of F - Dbar, 0 at a tie as in the FP64 definition
        const float g0 = __ldg(&gt[3 * p]), g1 = __ldg(&gt[3 * p + 1]), g2 = __ldg(&gt[3 * p + 2]);
        const float F = __ldg(&fused[p]);
        // every load of the pixel is issued before the sums (the views' alphas, then the
        // colours and depths of all views, covered or not): the pixel's K gathers overlap
        // instead of waiting on one another.  A view adds only where a_k = 1, in view order.
        constexpr int KB = 4;
        int A = 0;
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, ed = 0.0f;
        for (int kb = 0; kb < K; kb += KB) {
            uint8_t a[KB];
            float4 c[KB];
            float dk[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) a[j] = kb + j < K ? __ldg(&alpha[(size_t)(kb + j) * HWt + p]) : 0;
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                if (kb + j < K) {
                    c[j] = __ldg(&color[(size_t)(kb + j) * HWt + p]);
                    dk[j] = __ldg(&wdepth[(size_t)(kb + j) * HWt + p]);
                }
            }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                if (a[j]) {
                    e0 += c[j].x - g0;
                    e1 += c[j].y - g1;
                    e2 += c[j].z - g2;
                    ed += F - dk[j];
                    ++A;
                }
            }
        }
        unsigned cd = (unsigned)A;
        if (A > 0) {
            const float inv = 1.0f / (float)A;
            l1 += (fabsf(e0) + fabsf(e1) + fabsf(e2)) * inv;
            cd |= (sign2(e0) << 6) | (sign2(e1) << 8) | (sign2(e2) << 10);
            n += 1;
            cd |= 1u << 14;
            if (F > 0.0f) {
                ld += fabsf(ed) * inv;
                cd |= sign2(ed) << 12;
                cd |= 1u << 15;
            }
        }
        code[p] = cd;
    }
    // block sums in a fixed order: each warp by a shuffle tree, then the warps in order
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        l1 += __shfl_down_sync(0xffffffffu, l1, m);
        ld += __shfl_down_sync(0xffffffffu, ld, m);
        n += __shfl_down_sync(0xffffffffu, n, m);
    }
    if ((threadIdx.x & 31) == 0) {
        s_l1[threadIdx.x >> 5] = l1;
        s_ld[threadIdx.x >> 5] = ld;
        s_n[threadIdx.x >> 5] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial q = {0.0, 0.0, 0ull};
        for (int w = 0; w < BL_THREADS / 32; ++w) {
            q.l1 += (double)s_l1[w];
            q.ld += (double)s_ld[w];
            q.n += s_n[w];
        }
        partial[blockIdx.x] = q;
    }
}

// One block of RD_THREADS: thread t adds partials t, t + RD_THREADS, ... in order,
// then the threads' sums meet in a fixed shuffle tree per warp and the warps'
// sums in a fixed tree in warp 0 (the same order on every run: deterministic).
// Few threads: the block runs on one SM, whose FP64 rate is small, so the FP64
// adds are kept near one per partial.  loss = {L, L1, L_Depth}; scale = {s_rgb, s_d}.
constexpr int RD_THREADS = 128;

__device__ __forceinline__ void tree_sum(double &l1, double &ld, unsigned long long &n) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        l1 += __shfl_down_sync(0xffffffffu, l1, m);
        ld += __shfl_down_sync(0xffffffffu, ld, m);
        n += __shfl_down_sync(0xffffffffu, n, m);
    }
}

__global__ void __launch_bounds__(RD_THREADS) blend_loss_reduce(const Partial *__restrict__ partial, int nblocks,
                                                                 int K, int64_t HWt, float w_l1, float w_depth,
                                                                 double *__restrict__ loss, float *__restrict__ scale) {
    __shared__ double s_l1[RD_THREADS / 32], s_ld[RD_THREADS / 32];
    __shared__ unsigned long long s_n[RD_THREADS / 32];
    double l1 = 0.0, ld = 0.0;
    unsigned long long n = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 8 * RD_THREADS) {
        // eight loads in flight, then their sums in order
        Partial q[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int b = b0 + i * RD_THREADS + threadIdx.x;
            if (b < nblocks) q[i] = partial[b];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (b0 + i * RD_THREADS + threadIdx.x < nblocks) {
                l1 += q[i].l1;
                ld += q[i].ld;
                n += q[i].n;
            }
        }
    }
    tree_sum(l1, ld, n);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_l1[w] = l1;
        s_ld[w] = ld;
        s_n[w] = n;
    }
    __syncthreads();
    if (w == 0) {
        const bool has = lane < RD_THREADS / 32;
        l1 = has ? s_l1[lane] : 0.0;
        ld = has ? s_ld[lane] : 0.0;
        n = has ? s_n[lane] : 0ull;
        tree_sum(l1, ld, n);
        if (lane == 0) {
            const double nn = n > 0 ? (double)n : 1.0;
            const double L1 = l1 / (3.0 * nn), LD = ld / ((double)K * (double)HWt);
            loss[0] = (double)w_l1 * L1 + (double)w_depth * LD;
            loss[1] = L1;
            loss[2] = LD;
            scale[0] = (float)((double)w_l1 / (3.0 * nn));
            scale[1] = (float)((double)w_depth / ((double)K * (double)HWt));
        }
    }
}

// grad_loss: the upstream d(out)/dL on the device, or null for 1.  The gradient
// for an upstream of 1 is formed first and then multiplied, so the values are
// those of scaling the unit gradient afterwards.
__global__ void __launch_bounds__(BL_THREADS) blend_loss_grad(int64_t HWt, const unsigned *__restrict__ code,
                                                              const float *__restrict__ scale,
                                                              const float *__restrict__ grad_loss,
                                                              float4 *__restrict__ grad_pixel,
                                                              float *__restrict__ grad_fused) {
    const int64_t p = (int64_t)blockIdx.x * BL_THREADS + threadIdx.x;
    if (p >= HWt) return;
    const unsigned cd = code[p];
    const int A = (int)(cd & 63u);
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float gf = 0.0f;
    if (cd & (1u << 14)) {
        const float inv = 1.0f / (float)A, s = scale[0] * inv;
        g.x = s * unsign2((cd >> 6) & 3u);
        g.y = s * unsign2((cd >> 8) & 3u);
        g.z = s * unsign2((cd >> 10) & 3u);
        if (cd & (1u << 15)) {
            const float sd = unsign2((cd >> 12) & 3u);
            gf = scale[1] * sd;
            g.w = -gf * inv;
        }
    }
    if (grad_loss) {
        const float u = __ldg(grad_loss);
        g = make_float4(g.x * u, g.y * u, g.z * u, g.w * u);
        gf *= u;
    }
    if (grad_pixel) grad_pixel[p] = g;
    if (grad_fused) grad_fused[p] = gf;
}

}  // namespace

BlendLossLayout blend_loss_layout(int64_t HWt) {
    auto up = [](size_t n) { return (n + 255) / 256 * 256; };
    BlendLossLayout L;
    L.nblocks = (int)((HWt + BL_THREADS - 1) / BL_THREADS);
    size_t o = 0;
    L.off_code = o; o = up(o + (size_t)HWt * 4);
    L.off_partial = o; o = up(o + (size_t)L.nblocks * sizeof(Partial));
    L.off_scale = o; o = up(o + 2 * sizeof(float));
    L.total = o;
    return L;
}

cudaError_t launch_blend_loss(int K, int64_t HWt, const float4 *color, const uint8_t *alpha, const float *wdepth,
                              const float *fused, const float *gt, float w_l1, float w_depth, double *loss,
                              float4 *grad_pixel, float *grad_fused, char *ws, cudaStream_t st) {
    const BlendLossLayout L = blend_loss_layout(HWt);
    unsigned *code = reinterpret_cast<unsigned *>(ws + L.off_code);
    Partial *partial = reinterpret_cast<Partial *>(ws + L.off_partial);
    float *scale = reinterpret_cast<float *>(ws + L.off_scale);
    const int pb = pass_blocks(HWt);
    blend_loss_pass<<<pb, BL_THREADS, 0, st>>>(K, HWt, color, alpha, wdepth, fused, gt, code, partial);
    blend_loss_reduce<<<1, RD_THREADS, 0, st>>>(partial, pb, K, HWt, w_l1, w_depth, loss, scale);
    if (grad_pixel || grad_fused)
        blend_loss_grad<<<L.nblocks, BL_THREADS, 0, st>>>(HWt, code, scale, nullptr, grad_pixel, grad_fused);
    return cudaGetLastError();
}

cudaError_t launch_blend_loss_grad(int64_t HWt, const char *ws, const float *grad_loss, float4 *grad_pixel,
                                   float *grad_fused, cudaStream_t st) {
    const BlendLossLayout L = blend_loss_layout(HWt);
    blend_loss_grad<<<L.nblocks, BL_THREADS, 0, st>>>(HWt, reinterpret_cast<const unsigned *>(ws + L.off_code),
                                                      reinterpret_cast<const float *>(ws + L.off_scale), grad_loss,
                                                      grad_pixel, grad_fused);
    return cudaGetLastError();
}

}  // namespace gvs
