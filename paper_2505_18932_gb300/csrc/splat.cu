// Per-view forward splatting into the target camera with a depth test
// (Sec. 3.1, Supplement A.3), as a 64-bit z-buffer.
//
// Views are processed in groups of `slots` (the number of target-sized key
// buffers the workspace holds).  A slot is one Ht x Wt array of keys
// (bits(z) << 32 | source index): the smallest key is the nearest surface,
// ties going to the lower source index, so the result does not depend on the
// order in which atomics land.  At 1080p a slot is 16.6 MB, which stays
// resident in the 126 MB L2 between scatter and resolve.
//   clear   : fill every slot with ~0 (once per call)
//   scatter : one thread per source pixel, contract geometry, atomicMin on
//             every covered target pixel
//   resolve : one thread per target pixel and view: decode the key, gather
//             the winner's colour, write the outputs and reset the key to ~0
//             for the next group.
#include <math.h>

#include "gvs_internal.cuh"

namespace gvs {
namespace {

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }

// keys must be 16-byte aligned; n is the number of 64-bit keys.
__global__ void __launch_bounds__(256) clear_keys(unsigned long long *__restrict__ keys, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ulonglong2 ones = make_ulonglong2(~0ull, ~0ull);
    ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(keys);
    for (int64_t q = first; q < n / 2; q += stride) k2[q] = ones;
    if (first == 0 && (n & 1)) keys[n - 1] = ~0ull;
}

__global__ void __launch_bounds__(256) splat_scatter(const SplatArgs a, int k0, int kn) {
    const int64_t HW = (int64_t)a.W * a.H;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)kn * HW) return;
    const int kk = (int)(p / HW);
    const int k = k0 + kk;
    const int src = (int)(p - (int64_t)kk * HW);
    const int v = src / a.W;
    const int u = src - v * a.W;
    const float d = __ldg(&a.depth[(size_t)k * HW + src]);
    if (!valid_depth(d)) return;
    const float *A = a.v[k].xf.M;
    const float *c = a.v[k].xf.b;
    const float fu = (float)u, fv = (float)v;
    const float m0 = __fmaf_rn(A[0], fu, __fmaf_rn(A[1], fv, A[2]));
    const float m1 = __fmaf_rn(A[3], fu, __fmaf_rn(A[4], fv, A[5]));
    const float m2 = __fmaf_rn(A[6], fu, __fmaf_rn(A[7], fv, A[8]));
    const float h0 = __fmaf_rn(d, m0, c[0]);
    const float h1 = __fmaf_rn(d, m1, c[1]);
    const float h2 = __fmaf_rn(d, m2, c[2]);
    if (!(h2 > 1e-6f)) return;
    const float x = __fdiv_rn(h0, h2);
    const float y = __fdiv_rn(h1, h2);
    float lox, hix, loy, hiy;
    if (a.footprint) {
        const float rho = __fmul_rn(a.v[k].f_ratio, __fdiv_rn(d, h2));
        const float hw = fminf(fmaxf(__fmul_rn(0.5f, rho), 0.5f), a.max_hw);
        lox = ceilf(__fsub_rn(x, hw));
        hix = floorf(__fadd_rn(x, hw));
        loy = ceilf(__fsub_rn(y, hw));
        hiy = floorf(__fadd_rn(y, hw));
    } else {
        lox = hix = rintf(x);
        loy = hiy = rintf(y);
    }
    // clip with plain comparisons so that a NaN bound (overflowed geometry) skips the pixel
    if (lox < 0.0f) lox = 0.0f;
    if (loy < 0.0f) loy = 0.0f;
    if (hix > (float)(a.Wt - 1)) hix = (float)(a.Wt - 1);
    if (hiy > (float)(a.Ht - 1)) hiy = (float)(a.Ht - 1);
    if (!(lox <= hix) || !(loy <= hiy)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(h2) << 32) | (unsigned)src;
    unsigned long long *slot = a.keys + (size_t)kk * a.Wt * a.Ht;
    const int i0 = (int)lox, i1 = (int)hix, j0 = (int)loy, j1 = (int)hiy;
    for (int jj = j0; jj <= j1; ++jj)
        for (int ii = i0; ii <= i1; ++ii) atomicMin(&slot[(size_t)jj * a.Wt + ii], key);
}

__global__ void __launch_bounds__(256) splat_resolve(const SplatArgs a, int k0, int kn) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)kn * HWt) return;
    const int kk = (int)(p / HWt);
    const int k = k0 + kk;
    const int64_t t = p - (int64_t)kk * HWt;
    unsigned long long *slot = a.keys + (size_t)kk * HWt;
    const unsigned long long key = slot[t];
    slot[t] = ~0ull;  // ready for the next group of views
    const bool has = key != ~0ull;
    const int32_t w = has ? (int32_t)(uint32_t)(key & 0xffffffffull) : -1;
    const float z = has ? __uint_as_float((uint32_t)(key >> 32)) : 0.0f;
    const size_t o = (size_t)k * HWt + t;
    a.winner[o] = w;
    if (a.warped_rgba) a.warped_rgba[o] = has ? __ldg(&a.rgba[(size_t)k * a.W * a.H + w]) : 0u;
    if (a.warped_depth) a.warped_depth[o] = z;
    if (a.alpha) a.alpha[o] = (uint8_t)has;
    if (a.guided) a.guided[o] = (uint8_t)(has && fabsf(z - __ldg(&a.fused[t])) <= a.mu_guide);
}

}  // namespace

cudaError_t launch_splat(const SplatArgs &a, int K, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int64_t HW = (int64_t)a.W * a.H;
    const int slots = a.slots < K ? a.slots : K;
    {
        const int64_t n = HWt * slots;
        int64_t blocks = (n / 2 + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        clear_keys<<<(unsigned)blocks, 256, 0, st>>>(a.keys, n);
    }
    for (int k0 = 0; k0 < K; k0 += slots) {
        const int kn = (K - k0) < slots ? (K - k0) : slots;
        const int64_t ns = (int64_t)kn * HW;
        splat_scatter<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(a, k0, kn);
        const int64_t nt = (int64_t)kn * HWt;
        splat_resolve<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(a, k0, kn);
    }
    return cudaGetLastError();
}

}  // namespace gvs
