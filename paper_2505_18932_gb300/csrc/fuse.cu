// Image-based TSDF fusion in the target view (Supplement A.1, Eq. 3).
//
// Two kernels:
//  * weight_map: the confidence weight of Supplement A.1 depends only on the
//    sampled input pixel (nearest-pixel sampling), so it is computed once per
//    input pixel and packed with the depth as float2 (d, omega).  An invalid
//    pixel is stored as (0, 0): its signed distance is then below -1 and it
//    never contributes.  7x7 stencil over a shared-memory tile with halo.
//  * fuse: one thread per target pixel marches the D samples in registers,
//    one 8-byte gather per (sample, view), and stops at the first +/-
//    crossing.  Per-ray affine coefficients make each projection three FMAs.
#include <math.h>

#include "gvs_internal.cuh"

namespace gvs {
namespace {

constexpr int WM_TX = 32;
constexpr int WM_TY = 8;

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }

// R = window / 2.  Tile of WM_TX x WM_TY outputs; halo replicated at borders.
template <int R>
__global__ void __launch_bounds__(WM_TX *WM_TY) weight_map_kernel(const float *__restrict__ depth,
                                                                  float2 *__restrict__ dw, int W, int H,
                                                                  float mu, float wconst, float inv_w2) {
    constexpr int SW = WM_TX + 2 * R;
    constexpr int SH = WM_TY + 2 * R;
    __shared__ float tile[SH][SW];
    const int k = blockIdx.z;
    const float *dep = depth + (size_t)k * W * H;
    const int x0 = blockIdx.x * WM_TX - R;
    const int y0 = blockIdx.y * WM_TY - R;
    const int tid = threadIdx.y * WM_TX + threadIdx.x;
    for (int e = tid; e < SW * SH; e += WM_TX * WM_TY) {
        const int sy = e / SW, sx = e - sy * SW;
        const int gx = min(max(x0 + sx, 0), W - 1);
        const int gy = min(max(y0 + sy, 0), H - 1);
        const float d = __ldg(&dep[(size_t)gy * W + gx]);
        tile[sy][sx] = valid_depth(d) ? d : __int_as_float(0x7fc00000);  // NaN marks invalid
    }
    __syncthreads();
    const int x = blockIdx.x * WM_TX + threadIdx.x;
    const int y = blockIdx.y * WM_TY + threadIdx.y;
    if (x >= W || y >= H) return;
    const float dc = tile[threadIdx.y + R][threadIdx.x + R];
    float2 out = make_float2(0.0f, 0.0f);
    if (dc == dc) {  // valid centre
        float nu = 0.0f;
#pragma unroll
        for (int dy = 0; dy <= 2 * R; ++dy) {
#pragma unroll
            for (int dx = 0; dx <= 2 * R; ++dx) {
                // fminf returns mu for a NaN (invalid) neighbour: it counts mu^2
                const float t = fminf(fabsf(dc - tile[threadIdx.y + dy][threadIdx.x + dx]), mu);
                nu = fmaf(t, t, nu);
            }
        }
        const float w = nu > 0.0f ? fminf(wconst * rsqrtf(nu * inv_w2), 1.0f) : 1.0f;
        out = make_float2(dc, w);
    }
    dw[(size_t)k * W * H + (size_t)y * W + x] = out;
}

// Nearest integer (ties to even) of the exact real quotient num/den, den > 0.
// q = num * r with r ~ 1/den (relative error a few ulp) is within 0.01 of the
// quotient for any quotient that can land inside an image (|q| < 2^14 + 1);
// only when q sits within 0.01 of a half-integer is the decision re-taken
// from the signs of the exact residuals num - (n +/- 0.5) den (one rounding
// each in the FMA, which never changes a sign).
__device__ __forceinline__ int nearest_of_quotient(float num, float den, float r) {
    const float q = num * r;
    float n = rintf(q);
    if (fabsf(q - n) > 0.49f && fabsf(n) < 4194304.0f) {
        const float hi = __fmaf_rn(-(n + 0.5f), den, num);
        const float lo = __fmaf_rn(-(n - 0.5f), den, num);
        const bool odd = (__float2int_rz(n) & 1) != 0;
        if (hi > 0.0f || (hi == 0.0f && odd)) n += 1.0f;
        else if (lo < 0.0f || (lo == 0.0f && odd)) n -= 1.0f;
    }
    return __float2int_rz(n);
}

constexpr int FZ_TX = 16;
constexpr int FZ_TY = 8;

template <int KMAX>
__global__ void __launch_bounds__(FZ_TX *FZ_TY) fuse_kernel(const FuseArgs a) {
    const int i = blockIdx.x * FZ_TX + threadIdx.x;
    const int j = blockIdx.y * FZ_TY + threadIdx.y;
    if (i >= a.Wt || j >= a.Ht) return;
    const float fi = (float)i, fj = (float)j;
    float ax[KMAX], ay[KMAX], az[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < a.K) {
            const float *M = a.xf[k].M;
            ax[k] = __fmaf_rn(M[0], fi, __fmaf_rn(M[1], fj, M[2]));
            ay[k] = __fmaf_rn(M[3], fi, __fmaf_rn(M[4], fj, M[5]));
            az[k] = __fmaf_rn(M[6], fi, __fmaf_rn(M[7], fj, M[8]));
        }
    }
    const size_t plane = (size_t)a.W * a.H;
    float S_prev = 0.0f, W_prev = 0.0f, z_prev = 0.0f;
    float out = 0.0f;
    int idx = -1;
    for (int s = 0; s < a.D; ++s) {
        const float zs = __fmaf_rn((float)s, a.dz, a.zn);
        float S = 0.0f, Wsum = 0.0f;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < a.K) {
                const float hz = __fmaf_rn(zs, az[k], a.xf[k].b[2]);
                if (hz > 1e-6f) {
                    const float hx = __fmaf_rn(zs, ax[k], a.xf[k].b[0]);
                    const float hy = __fmaf_rn(zs, ay[k], a.xf[k].b[1]);
                    const float r = __fdividef(1.0f, hz);
                    const int u = nearest_of_quotient(hx, hz, r);
                    const int v = nearest_of_quotient(hy, hz, r);
                    if ((unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H) {
                        const float2 p = __ldg(&a.dw[(size_t)k * plane + (size_t)v * a.W + u]);
                        const float sdf = (p.x - hz) * a.inv_mu;
                        if (sdf >= -1.0f) {
                            S = fmaf(p.y, fminf(sdf, 1.0f), S);
                            Wsum += p.y;
                        }
                    }
                }
            }
        }
        if (a.normalize && Wsum > 0.0f) S = S / Wsum;
        if (s > 0 && W_prev > 0.0f && Wsum > 0.0f && S_prev > 0.0f && S <= 0.0f) {
            out = z_prev + (zs - z_prev) * (S_prev / (S_prev - S));
            idx = s - 1;
            break;
        }
        S_prev = S;
        W_prev = Wsum;
        z_prev = zs;
    }
    const size_t o = (size_t)j * a.Wt + i;
    a.fused[o] = out;
    if (a.crossing) a.crossing[o] = (int16_t)idx;
}

template <int R>
cudaError_t launch_wm(const float *depth, float2 *dw, int K, int W, int H, float mu, float wconst, float inv_w2,
                      cudaStream_t st) {
    dim3 grid((W + WM_TX - 1) / WM_TX, (H + WM_TY - 1) / WM_TY, K);
    weight_map_kernel<R><<<grid, dim3(WM_TX, WM_TY), 0, st>>>(depth, dw, W, H, mu, wconst, inv_w2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_weight_map(const float *depth, float2 *dw, int K, int W, int H, float mu, float wconst,
                              int window, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const float inv_w2 = (float)(1.0 / ((double)window * (double)window));
    switch (window / 2) {
        case 0: return launch_wm<0>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 1: return launch_wm<1>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 2: return launch_wm<2>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 3: return launch_wm<3>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 4: return launch_wm<4>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 5: return launch_wm<5>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 6: return launch_wm<6>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        case 7: return launch_wm<7>(depth, dw, K, W, H, mu, wconst, inv_w2, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fuse(const FuseArgs &a, cudaStream_t st) {
    dim3 grid((a.Wt + FZ_TX - 1) / FZ_TX, (a.Ht + FZ_TY - 1) / FZ_TY);
    dim3 block(FZ_TX, FZ_TY);
    if (a.K <= 4) fuse_kernel<4><<<grid, block, 0, st>>>(a);
    else if (a.K <= 8) fuse_kernel<8><<<grid, block, 0, st>>>(a);
    else if (a.K <= 16) fuse_kernel<16><<<grid, block, 0, st>>>(a);
    else fuse_kernel<32><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gvs
