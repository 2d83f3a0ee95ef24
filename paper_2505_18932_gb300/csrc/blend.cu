// Blending-network input and the blend of Eqs. 4-5 (Sec. 3.3; the
// supplement's list of network inputs).
//   features : one thread per target pixel writes the 9K + 1 channel planes
//              (rendered colours, their depths and alphas, the TSDF depth,
//              then per view n . d_k, r_t . d_k, |c_k - c_t|, z_k . z_t);
//              FP32 arithmetic, stored as FP32, FP16 or BF16.
//   blend    : one thread per target pixel, I = (1 - w_BG) I_FG + w_BG I_BG
//              with I_FG the alpha-and-weight normalised sum over views, and
//              per-block partial sums of |D - D_blend| for L_Depth, reduced
//              by one block in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "blend_internal.cuh"

namespace gvs {
namespace {

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }

__device__ __forceinline__ void store(float *p, float v) { *p = v; }
__device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float load(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename OT>
__global__ void __launch_bounds__(256) features_kernel(const BlendArgs a, OT *__restrict__ out) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i >= a.Wt || j >= a.Ht) return;
    const int K = a.K;
    const size_t np = (size_t)a.Wt * a.Ht;
    const size_t p = (size_t)j * a.Wt + i;
    for (int k = 0; k < K; ++k) {
        const size_t o = (size_t)k * np + p;
        const uint32_t c = __ldg(&a.rgba[o]);
        store(&out[(size_t)(3 * k + 0) * np + p], (float)(c & 0xffu) * (1.0f / 255.0f));
        store(&out[(size_t)(3 * k + 1) * np + p], (float)((c >> 8) & 0xffu) * (1.0f / 255.0f));
        store(&out[(size_t)(3 * k + 2) * np + p], (float)((c >> 16) & 0xffu) * (1.0f / 255.0f));
        store(&out[(size_t)(3 * K + k) * np + p], __ldg(&a.wdepth[o]));
        store(&out[(size_t)(4 * K + k) * np + p], (float)__ldg(&a.alpha[o]));
        store(&out[(size_t)(7 * K + 1 + k) * np + p], a.dist[k]);
        store(&out[(size_t)(8 * K + 1 + k) * np + p], a.axis[k]);
    }
    const float D = __ldg(&a.fused[p]);
    store(&out[(size_t)(5 * K) * np + p], D);
    const bool have = valid_depth(D);
    float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
    if (have && i > 0 && i < a.Wt - 1 && j > 0 && j < a.Ht - 1) {
        const float dl = __ldg(&a.fused[p - 1]), dr = __ldg(&a.fused[p + 1]);
        const float du = __ldg(&a.fused[p - a.Wt]), dd = __ldg(&a.fused[p + a.Wt]);
        if (valid_depth(dl) && valid_depth(dr) && valid_depth(du) && valid_depth(dd)) {
            // central differences of the back-projected points, written without
            // subtracting two large coordinates
            const float fi = (float)i - a.cx, fj = (float)j - a.cy;
            const float dh = dr - dl, sh = dr + dl, dv = dd - du, sv = dd + du;
            const float a0 = (dh * fi + sh) / a.fx, a1 = dh * fj / a.fy, a2 = dh;
            const float b0 = dv * fi / a.fx, b1 = (dv * fj + sv) / a.fy, b2 = dv;
            n0 = a1 * b2 - a2 * b1;
            n1 = a2 * b0 - a0 * b2;
            n2 = a0 * b1 - a1 * b0;
            const float P0 = D * fi / a.fx, P1 = D * fj / a.fy;
            if (n0 * P0 + n1 * P1 + n2 * D > 0.0f) {
                n0 = -n0;
                n1 = -n1;
                n2 = -n2;
            }
            const float l2 = n0 * n0 + n1 * n1 + n2 * n2;
            if (l2 > 0.0f) {
                const float inv = rsqrtf(l2);
                n0 *= inv;
                n1 *= inv;
                n2 *= inv;
            }
        }
    }
    float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f, rl = 0.0f;
    if (have) {
        P0 = D * ((float)i - a.cx) / a.fx;
        P1 = D * ((float)j - a.cy) / a.fy;
        P2 = D;
        rl = rsqrtf(P0 * P0 + P1 * P1 + P2 * P2);
    }
    for (int k = 0; k < K; ++k) {
        float nd = 0.0f, rd = 0.0f;
        if (have) {
            const float d0 = P0 - a.ck[k][0], d1 = P1 - a.ck[k][1], d2 = P2 - a.ck[k][2];
            const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            nd = (n0 * d0 + n1 * d1 + n2 * d2) * il;
            rd = (P0 * d0 + P1 * d1 + P2 * d2) * il * rl;
        }
        store(&out[(size_t)(5 * K + 1 + k) * np + p], nd);
        store(&out[(size_t)(6 * K + 1 + k) * np + p], rd);
    }
}

template <typename WT>
__global__ void __launch_bounds__(256) blend_kernel(const BlendArgs a, const WT *__restrict__ w,
                                                    const WT *__restrict__ w_bg, const WT *__restrict__ i_bg,
                                                    float *__restrict__ image, double *__restrict__ partial) {
    __shared__ float red[8];
    const int64_t np = (int64_t)a.Wt * a.Ht;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float ad = 0.0f;
    if (p < np) {
        float den = 0.0f, r = 0.0f, g = 0.0f, b = 0.0f, dn = 0.0f;
        for (int k = 0; k < a.K; ++k) {
            const size_t o = (size_t)k * np + p;
            const float aw = (float)__ldg(&a.alpha[o]) * load(&w[o]);
            const uint32_t c = __ldg(&a.rgba[o]);
            r = fmaf((float)(c & 0xffu) * (1.0f / 255.0f), aw, r);
            g = fmaf((float)((c >> 8) & 0xffu) * (1.0f / 255.0f), aw, g);
            b = fmaf((float)((c >> 16) & 0xffu) * (1.0f / 255.0f), aw, b);
            dn = fmaf(__ldg(&a.wdepth[o]), aw, dn);
            den += aw;
        }
        const float inv = den > 0.0f ? 1.0f / den : 0.0f;
        const float wb = load(&w_bg[p]);
        image[p] = (1.0f - wb) * (r * inv) + wb * load(&i_bg[p]);
        image[np + p] = (1.0f - wb) * (g * inv) + wb * load(&i_bg[np + p]);
        image[2 * np + p] = (1.0f - wb) * (b * inv) + wb * load(&i_bg[2 * np + p]);
        ad = fabsf(__ldg(&a.fused[p]) - dn * inv);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) ad += __shfl_xor_sync(0xffffffffu, ad, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += (double)red[q];
        partial[blockIdx.x] = s;
    }
}

// One block sums the per-block partials in a fixed order.
__global__ void __launch_bounds__(256) blend_reduce(const double *__restrict__ partial, int n, double scale,
                                                    double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) s += partial[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

}  // namespace

cudaError_t launch_blend_features(const BlendArgs &a, int out_dtype, void *out, cudaStream_t st) {
    const dim3 grid((unsigned)((a.Wt + 31) / 32), (unsigned)((a.Ht + 7) / 8)), block(32, 8);
    if (out_dtype == GVS_F16) features_kernel<__half><<<grid, block, 0, st>>>(a, reinterpret_cast<__half *>(out));
    else if (out_dtype == GVS_BF16)
        features_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(a, reinterpret_cast<__nv_bfloat16 *>(out));
    else features_kernel<float><<<grid, block, 0, st>>>(a, reinterpret_cast<float *>(out));
    return cudaGetLastError();
}

int blend_blocks(int Wt, int Ht) { return (int)(((int64_t)Wt * Ht + 255) / 256); }

cudaError_t launch_blend(const BlendArgs &a, int weight_dtype, const void *w, const void *w_bg, const void *i_bg,
                         float *image, double *l_depth, double *partial, cudaStream_t st) {
    const int nb = blend_blocks(a.Wt, a.Ht);
    if (weight_dtype == GVS_BF16)
        blend_kernel<__nv_bfloat16><<<nb, 256, 0, st>>>(a, reinterpret_cast<const __nv_bfloat16 *>(w),
                                                         reinterpret_cast<const __nv_bfloat16 *>(w_bg),
                                                         reinterpret_cast<const __nv_bfloat16 *>(i_bg), image, partial);
    else
        blend_kernel<float><<<nb, 256, 0, st>>>(a, reinterpret_cast<const float *>(w),
                                                reinterpret_cast<const float *>(w_bg),
                                                reinterpret_cast<const float *>(i_bg), image, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !l_depth) return e;
    blend_reduce<<<1, 256, 0, st>>>(partial, nb, 1.0 / ((double)a.Wt * a.Ht * a.K), l_depth);
    return cudaGetLastError();
}

}  // namespace gvs
