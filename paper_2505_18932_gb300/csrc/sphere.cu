// The paper's own raymarch for the image-based TSDF (Supplement A.1): from
// z_near, advance by 0.8 s until s changes sign, then three bisection steps.
// One thread per target ray; the per-view ray coefficients, the sample
// evaluation and the nearest-pixel contract are those of the uniform march
// (fuse_march.cuh).  Every operation that moves the march is an explicitly
// rounded FP32 operation and the weights come from the correctly rounded map,
// so the trajectory, the evaluation count and the depth are reproducible bit
// for bit on the host (see gvs_fuse_depth_sphere in gvs.h).
#include "fuse_march.cuh"
#include "sphere_internal.cuh"

namespace gvs {
namespace {

// evaluate_sample of the uniform march with a branch per view in place of the
// predicated gather: the same S and W.  Used when the call has fewer views than
// KMAX (the per-view guard already splits the code there, and the branches let
// lanes at unrelated depths skip work); with exactly KMAX views the predicated
// form, one block of code over all views, is faster (3.80 against 4.38 ms at
// 8 x 1080p).
template <int KMAX>
__device__ __forceinline__ void sphere_sample(const FuseArgs &a, const Ray (&ray)[KMAX], float zs, float &S,
                                              float &Wsum) {
    const float2 *map = reinterpret_cast<const float2 *>(a.dw);
    const size_t plane = (size_t)a.W * a.H;
    S = 0.0f;
    Wsum = 0.0f;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < a.K) {
            const float hz = __fmaf_rn(zs, ray[k].az, a.xf[k].b[2]);
            if (hz > 1e-6f) {
                const float hx = __fmaf_rn(zs, ray[k].ax, a.xf[k].b[0]);
                const float hy = __fmaf_rn(zs, ray[k].ay, a.xf[k].b[1]);
                int u, v;
                nearest_pixel(hx, hy, hz, u, v);
                if ((unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H &&
                    GVS_IN_BOUNDS((size_t)k * plane + (size_t)v * a.W + u, (size_t)a.K * plane, GVS_SITE_FUSE_MAP)) {
                    const float2 p = __ldg(&map[(size_t)k * plane + (size_t)v * a.W + u]);
                    const float sdf = (p.x - hz) * a.inv_mu;
                    if (sdf >= -1.0f) {
                        S = fmaf(p.y, fminf(sdf, 1.0f), S);
                        Wsum += p.y;
                    }
                }
            }
        }
    }
}

template <int KMAX, bool FULL>
__device__ __forceinline__ void sphere_eval(const FuseArgs &a, const Ray (&ray)[KMAX], float z, float &S, float &W) {
    if (FULL) evaluate_sample<KMAX, float2, true, true>(a, ray, z, S, W);
    else sphere_sample<KMAX>(a, ray, z, S, W);
}

// FULL: the call has exactly KMAX views.
template <int KMAX, bool FULL>
__global__ void __launch_bounds__(128) sphere_kernel(const __grid_constant__ SphereArgs s) {
    const FuseArgs &a = s.f;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    if (i >= a.Wt || j >= a.Ht) return;
    const float fi = (float)i, fj = (float)j;
    Ray ray[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (FULL || k < a.K) {
            const float *M = a.xf[k].M;
            ray[k].ax = __fmaf_rn(M[0], fi, __fmaf_rn(M[1], fj, M[2]));
            ray[k].ay = __fmaf_rn(M[3], fi, __fmaf_rn(M[4], fj, M[5]));
            ray[k].az = __fmaf_rn(M[6], fi, __fmaf_rn(M[7], fj, M[8]));
        }
    }
    float z = a.zn, z_prev = 0.0f, S_prev = 0.0f, W_prev = 0.0f, out = 0.0f;
    bool have_prev = false;
    int evals = 0;
    for (int it = 0; it < s.max_steps && z <= s.zf; ++it) {
        float S, W;
        sphere_eval<KMAX, FULL>(a, ray, z, S, W);
        ++evals;
        if (have_prev && W_prev > 0.0f && W > 0.0f && S_prev > 0.0f && S <= 0.0f) {
            float lo = z_prev, hi = z;
            for (int b = 0; b < 3; ++b) {
                const float m = __fmul_rn(0.5f, __fadd_rn(lo, hi));
                float Sm, Wm;
                sphere_eval<KMAX, FULL>(a, ray, m, Sm, Wm);
                ++evals;
                if (Wm > 0.0f && Sm > 0.0f) lo = m;
                else hi = m;
            }
            out = __fmul_rn(0.5f, __fadd_rn(lo, hi));
            break;
        }
        float stepn = 1.0f;
        if (W > 0.0f) {
            const float sn = __fdiv_rn(S, W);
            stepn = sn > s.min_frac ? sn : s.min_frac;
        }
        S_prev = S;
        W_prev = W;
        z_prev = z;
        have_prev = true;
        z = __fadd_rn(z, __fmul_rn(s.c08mu, stepn));
    }
    const size_t o = (size_t)j * a.Wt + i;
    a.fused[o] = out;
    if (s.evals) s.evals[o] = evals;
}

template <int KMAX>
void launch_k(const SphereArgs &s, cudaStream_t st) {
    const dim3 grid((unsigned)((s.f.Wt + 31) / 32), (unsigned)((s.f.Ht + 3) / 4)), block(32, 4);
    if (s.f.K == KMAX) sphere_kernel<KMAX, true><<<grid, block, 0, st>>>(s);
    else sphere_kernel<KMAX, false><<<grid, block, 0, st>>>(s);
}

}  // namespace

cudaError_t launch_sphere(const SphereArgs &s, cudaStream_t st) {
    if (s.f.K <= 4) launch_k<4>(s, st);
    else if (s.f.K <= 8) launch_k<8>(s, st);
    else if (s.f.K <= 16) launch_k<16>(s, st);
    else launch_k<32>(s, st);
    return cudaGetLastError();
}

GVS_BOUNDS_TAKE_FN(bounds_take_sphere)

}  // namespace gvs
