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
#include <cuda_fp16.h>
#include <math.h>

#include "bounds_check.cuh"
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

__device__ __forceinline__ float load_depth(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_depth(const __half *p) { return __half2float(__ldg(p)); }

// The FP32 address contract of one source pixel (see gvs.h): projected
// position, depth, footprint half-width and the covered target pixels.
struct Geo {
    bool ok;
    float x, y, z, hw, m0, m1, m2;
    int i0, i1, j0, j1;
};

__device__ __forceinline__ Geo contract(const SplatView &sv, int u, int v, float d, int Wt, int Ht, int footprint,
                                        float max_hw) {
    Geo g;
    g.ok = false;
    if (!valid_depth(d)) return g;
    const float *A = sv.xf.M;
    const float *c = sv.xf.b;
    const float fu = (float)u, fv = (float)v;
    g.m0 = __fmaf_rn(A[0], fu, __fmaf_rn(A[1], fv, A[2]));
    g.m1 = __fmaf_rn(A[3], fu, __fmaf_rn(A[4], fv, A[5]));
    g.m2 = __fmaf_rn(A[6], fu, __fmaf_rn(A[7], fv, A[8]));
    const float h0 = __fmaf_rn(d, g.m0, c[0]);
    const float h1 = __fmaf_rn(d, g.m1, c[1]);
    const float h2 = __fmaf_rn(d, g.m2, c[2]);
    if (!(h2 > 1e-6f)) return g;
    const float x = __fdiv_rn(h0, h2);
    const float y = __fdiv_rn(h1, h2);
    float lox, hix, loy, hiy, hw = 0.5f;
    if (footprint) {
        const float rho = __fmul_rn(sv.f_ratio, __fdiv_rn(d, h2));
        hw = fminf(fmaxf(__fmul_rn(0.5f, rho), 0.5f), max_hw);
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
    if (hix > (float)(Wt - 1)) hix = (float)(Wt - 1);
    if (hiy > (float)(Ht - 1)) hiy = (float)(Ht - 1);
    if (!(lox <= hix) || !(loy <= hiy)) return g;
    g.ok = true;
    g.x = x; g.y = y; g.z = h2; g.hw = hw;
    g.i0 = (int)lox; g.i1 = (int)hix; g.j0 = (int)loy; g.j1 = (int)hiy;
    return g;
}

// The covered target pixels of the contract above without its correctly
// rounded divisions.  The three quotients are taken with the fast approximate
// division (at most 2 ulp from the exact quotient for divisors in
// [2^-126, 2^126]); each bound is then an integer decision on a value within
// eps of the contract's own value.  The worst-case difference of x -/+ hw
// between the two: 2.5 ulp of the quotient x (2.98e-7 |x|), half of the
// difference of rho (its quotient 2.5 ulp plus both products' roundings:
// 4.2e-7 rho, so 4.2e-7 hw after the halving and the clamps) and the two
// roundings of the sum (1.2e-7 (|x| + hw)): at most 5.4e-7 (|x| + hw); the
// point mode's nearest pixel needs 3e-7 |x|.  With
//   eps = 1e-6 * (|x| + hw)   (1.85x that bound),
// a value further than eps from every decision boundary (an integer for
// ceil/floor, a half-integer for round-to-nearest) gives the contract's bound.
// Returns 1 (covered pixels in i0..j1), 0 (no pixel), or -1 when some value is
// within eps of a boundary or out of the fast division's range: the caller
// then evaluates the exact contract.  z is h2, computed exactly as there.
struct Bounds {
    int i0, i1, j0, j1;
    float z;
};

__device__ __forceinline__ float dist_to_integer(float t) { return fabsf(t - rintf(t)); }

__device__ __forceinline__ int contract_bounds_fast(const SplatView &sv, int u, int v, float d, int Wt, int Ht,
                                                    int footprint, float max_hw, Bounds &o) {
    if (!valid_depth(d)) return 0;
    const float *A = sv.xf.M;
    const float *c = sv.xf.b;
    const float fu = (float)u, fv = (float)v;
    const float m0 = __fmaf_rn(A[0], fu, __fmaf_rn(A[1], fv, A[2]));
    const float m1 = __fmaf_rn(A[3], fu, __fmaf_rn(A[4], fv, A[5]));
    const float m2 = __fmaf_rn(A[6], fu, __fmaf_rn(A[7], fv, A[8]));
    const float h0 = __fmaf_rn(d, m0, c[0]);
    const float h1 = __fmaf_rn(d, m1, c[1]);
    const float h2 = __fmaf_rn(d, m2, c[2]);
    if (!(h2 > 1e-6f)) return 0;
    if (!(h2 < 1e30f)) return -1;
    const float x = __fdividef(h0, h2);
    const float y = __fdividef(h1, h2);
    // far outside any target (|x| < 2^22 keeps eps below one pixel), or NaN: exact path
    if (!(fabsf(x) < 4.0e6f) || !(fabsf(y) < 4.0e6f)) return -1;
    float lox, hix, loy, hiy;
    if (footprint) {
        const float rho = __fmul_rn(sv.f_ratio, __fdividef(d, h2));
        const float hw = fminf(fmaxf(__fmul_rn(0.5f, rho), 0.5f), max_hw);
        const float a0 = __fsub_rn(x, hw), a1 = __fadd_rn(x, hw);
        const float b0 = __fsub_rn(y, hw), b1 = __fadd_rn(y, hw);
        const float ex = 1e-6f * (fabsf(x) + hw) + 1e-30f;
        const float ey = 1e-6f * (fabsf(y) + hw) + 1e-30f;
        if (!(fminf(dist_to_integer(a0), dist_to_integer(a1)) > ex) ||
            !(fminf(dist_to_integer(b0), dist_to_integer(b1)) > ey))
            return -1;
        lox = ceilf(a0);
        hix = floorf(a1);
        loy = ceilf(b0);
        hiy = floorf(b1);
    } else {
        const float ex = 1e-6f * fabsf(x) + 1e-30f, ey = 1e-6f * fabsf(y) + 1e-30f;
        if (!(dist_to_integer(__fsub_rn(x, 0.5f)) > ex) || !(dist_to_integer(__fsub_rn(y, 0.5f)) > ey))
            return -1;
        lox = hix = rintf(x);
        loy = hiy = rintf(y);
    }
    if (lox < 0.0f) lox = 0.0f;
    if (loy < 0.0f) loy = 0.0f;
    if (hix > (float)(Wt - 1)) hix = (float)(Wt - 1);
    if (hiy > (float)(Ht - 1)) hiy = (float)(Ht - 1);
    if (!(lox <= hix) || !(loy <= hiy)) return 0;
    o.i0 = (int)lox; o.i1 = (int)hix; o.j0 = (int)loy; o.j1 = (int)hiy;
    o.z = h2;
    return 1;
}

// Block of 32 x 8 source pixels, grid (ceil(W / 32), ceil(H / 8), views of
// the group): view, row and column come from the block coordinates, so no
// integer division.  DT: float or __half depth storage, widened to FP32.
// REJECT: candidates in front of the fused surface (z < fused - mu_guide)
// take no part in the depth test.
constexpr int SC_BX = 32, SC_BY = 8;

template <typename DT, bool REJECT = false>
__global__ void __launch_bounds__(SC_BX * SC_BY) splat_scatter(const SplatArgs a, int k0) {
    const int u = blockIdx.x * SC_BX + threadIdx.x;
    const int v = blockIdx.y * SC_BY + threadIdx.y;
    if (u >= a.W || v >= a.H) return;
    const int kk = blockIdx.z;
    const int k = k0 + kk;
    const int src = v * a.W + u;
    const float d = load_depth(reinterpret_cast<const DT *>(a.depth) + (size_t)k * a.W * a.H + src);
    Bounds b;
    int ok = contract_bounds_fast(a.v[k], u, v, d, a.Wt, a.Ht, a.footprint, a.max_hw, b);
    if (ok < 0) {
        const Geo g = contract(a.v[k], u, v, d, a.Wt, a.Ht, a.footprint, a.max_hw);
        ok = g.ok;
        b.i0 = g.i0; b.i1 = g.i1; b.j0 = g.j0; b.j1 = g.j1; b.z = g.z;
    }
    if (!ok) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(b.z) << 32) | (unsigned)src;
    unsigned long long *slot = a.keys + (size_t)kk * a.Wt * a.Ht;
    if (b.j1 - b.j0 <= 1 && b.i1 - b.i0 <= 1) {
        // the usual pixel-sized footprint: at most 2 x 2 pixels, one predicated body
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int jj = b.j0 + (e >> 1), ii = b.i0 + (e & 1);
            if (jj <= b.j1 && ii <= b.i1) {
                const size_t t = (size_t)jj * a.Wt + ii;
                if (!GVS_IN_BOUNDS(t, (size_t)a.Wt * a.Ht, GVS_SITE_SPLAT_KEY)) continue;
                if (REJECT && b.z < __fsub_rn(__ldg(&a.fused[t]), a.mu_guide)) continue;
                atomicMin(&slot[t], key);
            }
        }
        return;
    }
    for (int jj = b.j0; jj <= b.j1; ++jj)
        for (int ii = b.i0; ii <= b.i1; ++ii) {
            const size_t t = (size_t)jj * a.Wt + ii;
            if (!GVS_IN_BOUNDS(t, (size_t)a.Wt * a.Ht, GVS_SITE_SPLAT_KEY)) continue;
            if (REJECT && b.z < __fsub_rn(__ldg(&a.fused[t]), a.mu_guide)) continue;
            atomicMin(&slot[t], key);
        }
}

inline dim3 scatter_grid(int W, int H, int kn) {
    return dim3((unsigned)((W + SC_BX - 1) / SC_BX), (unsigned)((H + SC_BY - 1) / SC_BY), (unsigned)kn);
}

__device__ __forceinline__ void decode(unsigned long long key, bool &has, int32_t &w, float &z) {
    has = key != ~0ull;
    w = has ? (int32_t)(uint32_t)(key & 0xffffffffull) : -1;
    z = has ? __uint_as_float((uint32_t)(key >> 32)) : 0.0f;
}

// One thread per target pixel and view (any size); grid (ceil(Wt Ht / 256), views of the group).
__global__ void __launch_bounds__(256) splat_resolve(const SplatArgs a, int k0) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= HWt) return;
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    unsigned long long *slot = a.keys + (size_t)kk * HWt;
    const unsigned long long key = slot[t];
    slot[t] = ~0ull;  // ready for the next group of views
    bool has;
    int32_t w;
    float z;
    decode(key, has, w, z);
    const size_t o = (size_t)k * HWt + t;
    a.winner[o] = w;
    if (a.warped_rgba) a.warped_rgba[o] = has ? __ldg(&a.rgba[(size_t)k * a.W * a.H + w]) : 0u;
    if (a.warped_depth) a.warped_depth[o] = z;
    if (a.alpha) a.alpha[o] = (uint8_t)has;
    if (a.guided) a.guided[o] = (uint8_t)(has && fabsf(z - __ldg(&a.fused[t])) <= a.mu_guide);
}

// P consecutive target pixels per thread (P = 4 or 8), every access a 16-byte
// (or, for the byte maps, 4-byte) vector; needs Wt * Ht divisible by P.  The
// P colour gathers are independent, so each thread keeps P in flight (eight
// per thread measured 6 us faster than four over 8 views at 1080p).
// Grid (ceil(Wt Ht / (256 P)), views of the group).
template <int P>
__global__ void __launch_bounds__(256) splat_resolveP(const SplatArgs a, int k0) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int qn = (int)(HWt / P);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= qn) return;
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    ulonglong2 *slot = reinterpret_cast<ulonglong2 *>(a.keys + (size_t)kk * HWt) + (size_t)t * (P / 2);
    ulonglong2 kv[P / 2];
#pragma unroll
    for (int q = 0; q < P / 2; ++q) kv[q] = slot[q];
    float4 f[P / 4];
    if (a.guided) {
#pragma unroll
        for (int q = 0; q < P / 4; ++q) f[q] = __ldg(reinterpret_cast<const float4 *>(a.fused) + (size_t)t * (P / 4) + q);
    }
#pragma unroll
    for (int q = 0; q < P / 2; ++q) slot[q] = make_ulonglong2(~0ull, ~0ull);
    bool h[P];
    int w[P];
    float z[P];
#pragma unroll
    for (int q = 0; q < P / 2; ++q) {
        decode(kv[q].x, h[2 * q], w[2 * q], z[2 * q]);
        decode(kv[q].y, h[2 * q + 1], w[2 * q + 1], z[2 * q + 1]);
    }
    uint32_t c[P];
    if (a.warped_rgba) {
        const uint32_t *src = a.rgba + (size_t)k * a.W * a.H;
#pragma unroll
        for (int q = 0; q < P; ++q)
            c[q] = (h[q] && GVS_IN_BOUNDS(w[q], (size_t)a.W * a.H, GVS_SITE_SPLAT_SRC)) ? __ldg(&src[w[q]]) : 0u;
    }
    const size_t o4 = ((size_t)k * HWt) / 4 + (size_t)t * (P / 4);
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
        __stcs(reinterpret_cast<int4 *>(a.winner) + o4 + q, make_int4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]));
        if (a.warped_rgba)
            __stcs(reinterpret_cast<uint4 *>(a.warped_rgba) + o4 + q,
                   make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
        if (a.warped_depth)
            __stcs(reinterpret_cast<float4 *>(a.warped_depth) + o4 + q,
                   make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]));
        if (a.alpha)
            __stcs(reinterpret_cast<unsigned int *>(a.alpha) + o4 + q,
                   (unsigned)h[4 * q] | ((unsigned)h[4 * q + 1] << 8) | ((unsigned)h[4 * q + 2] << 16) |
                       ((unsigned)h[4 * q + 3] << 24));
        if (a.guided) {
            const unsigned g0 = h[4 * q] && fabsf(z[4 * q] - f[q].x) <= a.mu_guide;
            const unsigned g1 = h[4 * q + 1] && fabsf(z[4 * q + 1] - f[q].y) <= a.mu_guide;
            const unsigned g2 = h[4 * q + 2] && fabsf(z[4 * q + 2] - f[q].z) <= a.mu_guide;
            const unsigned g3 = h[4 * q + 3] && fabsf(z[4 * q + 3] - f[q].w) <= a.mu_guide;
            __stcs(reinterpret_cast<unsigned int *>(a.guided) + o4 + q, g0 | (g1 << 8) | (g2 << 16) | (g3 << 24));
        }
    }
}

// 256-bit global accesses (sm_100 and later): the address must be 32-byte aligned.
__device__ __forceinline__ void ld256(const unsigned long long *p, unsigned long long (&v)[4]) {
    asm volatile("ld.global.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
}
__device__ __forceinline__ void st256_ones(unsigned long long *p) {
    const unsigned long long o = ~0ull;
    asm volatile("st.global.v4.u64 [%0], {%1, %1, %1, %1};" ::"l"(p), "l"(o) : "memory");
}
__device__ __forceinline__ void st256_cs(void *p, const uint32_t (&v)[8]) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

inline bool aligned_to(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// ---- TMA bulk copies (cp.async.bulk) and the mbarrier that completes them ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bulk copies that did not complete within the wait limit (a status of the
// library, read and cleared by gvs_take_device_status).
__device__ unsigned g_async_timeouts = 0;

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
// Waits for phase 0 of the barrier, at most ~2^24 polls; false when it gave up.
__device__ __forceinline__ bool wait_phase0(uint32_t bar) {
    for (int i = 0; i < (1 << 24); ++i) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// The resolve with its streams moved by TMA: per block 1024 consecutive target
// pixels of one view.  One thread loads the block's keys (and fused depths) into
// shared memory with bulk copies completed on an mbarrier; every thread decodes
// four pixels (strided, so a warp reads 32 consecutive keys), gathers their
// winners' colours and writes the outputs into shared memory; one thread then
// stores the five outputs and the reset keys (~0) with bulk copies.  Only the
// colour gathers are per-thread global loads.  Needs Wt * Ht divisible by 16
// and every array 16-byte aligned (the caller checks).  Grid (ceil(Wt Ht /
// 1024), views of the group).
constexpr int RT_PX = 1024;
__global__ void __launch_bounds__(256) splat_resolve_tma(const SplatArgs a, int k0) {
    __shared__ __align__(128) unsigned long long s_key[RT_PX];
    __shared__ __align__(128) float s_fused[RT_PX];
    __shared__ __align__(128) int32_t s_win[RT_PX];
    __shared__ __align__(128) uint32_t s_rgba[RT_PX];
    __shared__ __align__(128) float s_dep[RT_PX];
    __shared__ __align__(128) uint8_t s_alpha[RT_PX];
    __shared__ __align__(128) uint8_t s_guided[RT_PX];
    __shared__ __align__(8) unsigned long long s_bar;
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int64_t base = (int64_t)blockIdx.x * RT_PX;
    const int n = (int)min((int64_t)RT_PX, HWt - base);
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    unsigned long long *slot = a.keys + (size_t)kk * HWt + base;
    const uint32_t bar = smem_addr(&s_bar);
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t kb = (uint32_t)n * 8u, fb = a.guided ? (uint32_t)n * 4u : 0u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kb + fb) : "memory");
        bulk_load(s_key, slot, kb, bar);
        if (a.guided) bulk_load(s_fused, a.fused + base, fb, bar);
    }
    if (!__syncthreads_and(wait_phase0(bar))) {  // the same answer in every thread
        if (tid == 0) atomicAdd(&g_async_timeouts, 1u);
        wait_phase0(bar);  // the copies may still land in this block's shared memory: give them time
        return;
    }
    const uint32_t *src = a.rgba + (size_t)k * a.W * a.H;
    uint32_t c[RT_PX / 256];
    int32_t wv[RT_PX / 256];
#pragma unroll
    for (int q = 0; q < RT_PX / 256; ++q) {
        const int p = q * 256 + tid;
        wv[q] = -1;
        c[q] = 0u;
        if (p < n) {
            bool h;
            float z;
            decode(s_key[p], h, wv[q], z);
            s_key[p] = ~0ull;  // ready for the next group of views
            s_win[p] = wv[q];
            s_dep[p] = z;
            s_alpha[p] = (uint8_t)h;
            if (a.guided) s_guided[p] = (uint8_t)(h && fabsf(z - s_fused[p]) <= a.mu_guide);
            if (a.warped_rgba && h && GVS_IN_BOUNDS(wv[q], (size_t)a.W * a.H, GVS_SITE_SPLAT_SRC))
                c[q] = __ldg(&src[wv[q]]);
        }
    }
    if (a.warped_rgba) {
#pragma unroll
        for (int q = 0; q < RT_PX / 256; ++q)
            if (q * 256 + tid < n) s_rgba[q * 256 + tid] = c[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // shared writes -> the bulk copies
    __syncthreads();
    if (tid == 0) {
        const size_t o = (size_t)k * HWt + base;
        bulk_store(a.winner + o, s_win, (uint32_t)n * 4u);
        if (a.warped_rgba) bulk_store(a.warped_rgba + o, s_rgba, (uint32_t)n * 4u);
        if (a.warped_depth) bulk_store(a.warped_depth + o, s_dep, (uint32_t)n * 4u);
        if (a.alpha) bulk_store(a.alpha + o, s_alpha, (uint32_t)n);
        if (a.guided) bulk_store(a.guided + o, s_guided, (uint32_t)n);
        bulk_store(slot, s_key, (uint32_t)n * 8u);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

// The TMA resolve applies: every bulk copy starts 16-byte aligned and moves a
// multiple of 16 bytes (1-byte planes: Wt * Ht divisible by 16).
inline bool tma_resolve_ok(const SplatArgs &a, int64_t HWt) {
    return HWt % 16 == 0 && aligned16(a.keys) && aligned16(a.winner) && aligned16(a.rgba) &&
           (!a.warped_rgba || aligned16(a.warped_rgba)) && (!a.warped_depth || aligned16(a.warped_depth)) &&
           (!a.alpha || aligned16(a.alpha)) && (!a.guided || (aligned16(a.guided) && a.fused && aligned16(a.fused)));
}

// ---------------------------------------------------------------------------
// Differentiable colour splat.  The hard z-buffer (scatter above) fixes the
// winner's depth z_w per target pixel; every covering source q inside the
// front band z_q <= z_w + mu_band adds a Gaussian weight
// g = exp(-|(x_q, y_q) - p|^2 / (2 sigma^2)), sigma = hw / 2 (a pixel-sized
// Gaussian, Sec. 3.1 / Supplement A.3), and the colour is sum g c / sum g.
// The adjoint gathers from the source side (one thread per source pixel
// walking its own footprint), so it needs no atomics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 load_color(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ float4 load_color(const uint2 *p) {  // four bfloat16
    const uint2 r = __ldg(p);
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                       __uint_as_float(r.y & 0xffff0000u));
}

// Grid as splat_scatter: blocks of 32 x 8 source pixels, z = view of the group.
// Its key loads (before the band test) wait on memory: eight resident blocks per
// SM (32 registers, no spill) against six at 39 registers, 26.0 -> 21.4 us a view.
template <typename DT, typename CT>
__global__ void __launch_bounds__(SC_BX * SC_BY, 8) soft_accum(const SplatArgs a, int k0) {
    const int64_t HW = (int64_t)a.W * a.H;
    const int u = blockIdx.x * SC_BX + threadIdx.x;
    const int v = blockIdx.y * SC_BY + threadIdx.y;
    if (u >= a.W || v >= a.H) return;
    const int kk = blockIdx.z;
    const int k = k0 + kk;
    const int src = v * a.W + u;
    const float d = load_depth(reinterpret_cast<const DT *>(a.depth) + (size_t)k * HW + src);
    const Geo g = contract(a.v[k], u, v, d, a.Wt, a.Ht, 1, a.max_hw);
    if (!g.ok) return;
    const float4 c = load_color(reinterpret_cast<const CT *>(a.color) + (size_t)k * HW + src);
    const float inv2s2 = 2.0f / (g.hw * g.hw);  // 1 / (2 sigma^2), sigma = hw / 2
    const unsigned long long *keys = a.keys + (size_t)kk * a.Wt * a.Ht;
    float4 *acc = a.acc + (size_t)kk * a.Wt * a.Ht;
    for (int jj = g.j0; jj <= g.j1; ++jj)
        for (int ii = g.i0; ii <= g.i1; ++ii) {
            const size_t t = (size_t)jj * a.Wt + ii;
            if (!GVS_IN_BOUNDS(t, (size_t)a.Wt * a.Ht, GVS_SITE_SOFT_ACC)) continue;
            const float zw = __uint_as_float((uint32_t)(keys[t] >> 32));
            if (!(g.z <= __fadd_rn(zw, a.mu_band))) continue;
            const float ex = g.x - (float)ii, ey = g.y - (float)jj;
            const float w = expf(-(ex * ex + ey * ey) * inv2s2);
            atomicAdd(&acc[t], make_float4(w * c.x, w * c.y, w * c.z, w));
        }
}

// One thread per target pixel (any size); grid (ceil(Wt Ht / 256), views of the group).
__global__ void __launch_bounds__(256) soft_resolve(const SplatArgs a, int k0) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= HWt) return;
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    unsigned long long *slot = a.keys + (size_t)kk * HWt;
    float4 *acc = a.acc + (size_t)kk * HWt;
    const unsigned long long key = slot[t];
    const float4 s = acc[t];
    slot[t] = ~0ull;  // ready for the next group of views
    acc[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool has;
    int32_t w;
    float z;
    decode(key, has, w, z);
    const size_t o = (size_t)k * HWt + t;
    a.winner[o] = w;
    if (a.warped_depth) a.warped_depth[o] = z;
    if (a.alpha) a.alpha[o] = (uint8_t)has;
    a.wsum[o] = s.w;
    const float r = (has && s.w > 0.0f) ? 1.0f / s.w : 0.0f;
    a.out_color[o] = make_float4(s.x * r, s.y * r, s.z * r, 0.0f);
}

// Four consecutive target pixels per thread, every access a 16-byte (bytes:
// 4-byte) vector; needs Wt * Ht divisible by 4.  Grid (ceil(Wt Ht / 1024), views).
__global__ void __launch_bounds__(256) soft_resolve4(const SplatArgs a, int k0) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int t4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t4 >= (int)(HWt / 4)) return;
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    ulonglong2 *slot = reinterpret_cast<ulonglong2 *>(a.keys + (size_t)kk * HWt) + 2 * (size_t)t4;
    float4 *acc = a.acc + (size_t)kk * HWt + 4 * (size_t)t4;
    const ulonglong2 k01 = slot[0], k23 = slot[1];
    float4 s[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] = acc[q];
    slot[0] = make_ulonglong2(~0ull, ~0ull);  // ready for the next group of views
    slot[1] = make_ulonglong2(~0ull, ~0ull);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool h[4];
    int32_t w[4];
    float z[4];
    decode(k01.x, h[0], w[0], z[0]);
    decode(k01.y, h[1], w[1], z[1]);
    decode(k23.x, h[2], w[2], z[2]);
    decode(k23.y, h[3], w[3], z[3]);
    const size_t o4 = ((size_t)k * HWt) / 4 + t4;
    __stcs(reinterpret_cast<int4 *>(a.winner) + o4, make_int4(w[0], w[1], w[2], w[3]));
    if (a.warped_depth) __stcs(reinterpret_cast<float4 *>(a.warped_depth) + o4, make_float4(z[0], z[1], z[2], z[3]));
    if (a.alpha)
        __stcs(reinterpret_cast<unsigned int *>(a.alpha) + o4,
               (unsigned)h[0] | ((unsigned)h[1] << 8) | ((unsigned)h[2] << 16) | ((unsigned)h[3] << 24));
    __stcs(reinterpret_cast<float4 *>(a.wsum) + o4, make_float4(s[0].w, s[1].w, s[2].w, s[3].w));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float r = (h[q] && s[q].w > 0.0f) ? 1.0f / s[q].w : 0.0f;
        __stcs(a.out_color + 4 * o4 + q, make_float4(s[q].x * r, s[q].y * r, s[q].z * r, 0.0f));
    }
}

__device__ __forceinline__ void ld256f(const float4 *p, float4 &x, float4 &y) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w), "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                 : "l"(p));
}
__device__ __forceinline__ void st256_zero(void *p) {
    const unsigned long long z = 0ull;
    asm volatile("st.global.v4.u64 [%0], {%1, %1, %1, %1};" ::"l"(p), "l"(z) : "memory");
}
__device__ __forceinline__ void st256f_cs(float4 *p, const float4 &x, const float4 &y) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(x.x), "f"(x.y),
                 "f"(x.z), "f"(x.w), "f"(y.x), "f"(y.y), "f"(y.z), "f"(y.w)
                 : "memory");
}

// Eight consecutive target pixels per thread with 32-byte accesses (20 memory
// instructions for 8 pixels instead of 40).  Needs Wt * Ht divisible by 8, the
// keys, accumulators, winner, depth, weight-sum and colour arrays 32-byte aligned
// and alpha 8-byte aligned (the caller checks).  Grid (ceil(Wt Ht / 2048), views).
__global__ void __launch_bounds__(256) soft_resolve_wide(const SplatArgs a, int k0) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int)(HWt / 8)) return;
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    unsigned long long *slot = a.keys + (size_t)kk * HWt + (size_t)t * 8;
    float4 *acc = a.acc + (size_t)kk * HWt + (size_t)t * 8;
    unsigned long long kv[8];
    {
        unsigned long long lo[4], hi[4];
        ld256(slot, lo);
        ld256(slot + 4, hi);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            kv[q] = lo[q];
            kv[4 + q] = hi[q];
        }
    }
    float4 sm[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) ld256f(acc + 2 * q, sm[2 * q], sm[2 * q + 1]);
    st256_ones(slot);  // ready for the next group of views
    st256_ones(slot + 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) st256_zero(acc + 2 * q);
    bool h[8];
    int32_t w[8];
    float z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) decode(kv[q], h[q], w[q], z[q]);
    const size_t o = (size_t)k * HWt + (size_t)t * 8;
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (uint32_t)w[q];
    st256_cs(a.winner + o, v);
    if (a.warped_depth) {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __float_as_uint(z[q]);
        st256_cs(a.warped_depth + o, v);
    }
    if (a.alpha) {
        unsigned long long m = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) m |= (unsigned long long)h[q] << (8 * q);
        __stcs(reinterpret_cast<unsigned long long *>(a.alpha + o), m);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __float_as_uint(sm[q].w);
    st256_cs(a.wsum + o, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 c[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float4 x = sm[2 * q + e];
            const float r = (h[2 * q + e] && x.w > 0.0f) ? 1.0f / x.w : 0.0f;
            c[e] = make_float4(x.x * r, x.y * r, x.z * r, 0.0f);
        }
        st256f_cs(a.out_color + o + 2 * q, c[0], c[1]);
    }
}

// The differentiable splat's resolve with its streams moved by TMA: per block
// 512 consecutive target pixels of one view.  One thread bulk-copies the keys
// and the (sum g c, sum g) accumulators into shared memory (mbarrier, bounded
// wait); every thread resolves two pixels (strided) and writes the winner,
// depth, alpha, weight sum and colour into shared memory and clears the keys
// (to ~0) and accumulators (to 0) in place; one thread bulk-stores the five
// outputs and the two resets.  Needs Wt * Ht divisible by 16 and every array
// 16-byte aligned (the caller checks).  Grid (ceil(Wt Ht / 512), views of the group).
constexpr int ST_PX = 512;
__global__ void __launch_bounds__(256) soft_resolve_tma(const SplatArgs a, int k0) {
    __shared__ __align__(128) unsigned long long s_key[ST_PX];
    __shared__ __align__(128) float4 s_acc[ST_PX];
    __shared__ __align__(128) int32_t s_win[ST_PX];
    __shared__ __align__(128) float s_dep[ST_PX];
    __shared__ __align__(128) float s_wsum[ST_PX];
    __shared__ __align__(128) float4 s_col[ST_PX];
    __shared__ __align__(128) uint8_t s_alpha[ST_PX];
    __shared__ __align__(8) unsigned long long s_bar;
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int64_t base = (int64_t)blockIdx.x * ST_PX;
    const int n = (int)min((int64_t)ST_PX, HWt - base);
    const int kk = blockIdx.y;
    const int k = k0 + kk;
    unsigned long long *slot = a.keys + (size_t)kk * HWt + base;
    float4 *acc = a.acc + (size_t)kk * HWt + base;
    const uint32_t bar = smem_addr(&s_bar);
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t kb = (uint32_t)n * 8u, ab = (uint32_t)n * 16u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kb + ab) : "memory");
        bulk_load(s_key, slot, kb, bar);
        bulk_load(s_acc, acc, ab, bar);
    }
    if (!__syncthreads_and(wait_phase0(bar))) {  // the same answer in every thread
        if (tid == 0) atomicAdd(&g_async_timeouts, 1u);
        wait_phase0(bar);  // the copies may still land in this block's shared memory: give them time
        return;
    }
#pragma unroll
    for (int q = 0; q < ST_PX / 256; ++q) {
        const int p = q * 256 + tid;
        if (p < n) {
            bool h;
            int32_t w;
            float z;
            decode(s_key[p], h, w, z);
            const float4 sm = s_acc[p];
            s_key[p] = ~0ull;  // ready for the next group of views
            s_acc[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            s_win[p] = w;
            s_dep[p] = z;
            s_alpha[p] = (uint8_t)h;
            s_wsum[p] = sm.w;
            const float r = (h && sm.w > 0.0f) ? 1.0f / sm.w : 0.0f;
            s_col[p] = make_float4(sm.x * r, sm.y * r, sm.z * r, 0.0f);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // shared writes -> the bulk copies
    __syncthreads();
    if (tid == 0) {
        const size_t o = (size_t)k * HWt + base;
        bulk_store(a.winner + o, s_win, (uint32_t)n * 4u);
        if (a.warped_depth) bulk_store(a.warped_depth + o, s_dep, (uint32_t)n * 4u);
        if (a.alpha) bulk_store(a.alpha + o, s_alpha, (uint32_t)n);
        bulk_store(a.wsum + o, s_wsum, (uint32_t)n * 4u);
        bulk_store(a.out_color + o, s_col, (uint32_t)n * 16u);
        bulk_store(slot, s_key, (uint32_t)n * 8u);
        bulk_store(acc, s_acc, (uint32_t)n * 16u);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

inline bool tma_soft_resolve_ok(const SplatArgs &a, int64_t HWt) {
    return HWt % 16 == 0 && aligned16(a.keys) && aligned16(a.acc) && aligned16(a.winner) &&
           (!a.warped_depth || aligned16(a.warped_depth)) && aligned16(a.wsum) && aligned16(a.out_color) &&
           (!a.alpha || aligned16(a.alpha));
}

inline bool wide_soft_resolve_ok(const SplatArgs &a, int64_t HWt) {
    return HWt % 8 == 0 && aligned_to(a.keys, 32) && aligned_to(a.acc, 32) && aligned_to(a.winner, 32) &&
           (!a.warped_depth || aligned_to(a.warped_depth, 32)) && aligned_to(a.wsum, 32) &&
           aligned_to(a.out_color, 32) && (!a.alpha || aligned_to(a.alpha, 8));
}

// Grid as splat_scatter over all views: blocks of 32 x 8 source pixels, z = view.
// Its footprint gathers wait on memory, so the kernel is built for eight resident
// blocks per SM (32 registers; a few values spill to L1): 403 -> 311 us for the
// 8 x 1080p views against five blocks at 48 registers.  BLENDED: the upstream
// gradient is one float4 per target pixel shared by every view (grad_pixel);
// otherwise per view (grad_color, grad_depth or null).
template <typename DT, typename CT, bool BLENDED>
__global__ void __launch_bounds__(SC_BX * SC_BY, 8) soft_bwd(const SplatArgs a) {
    const int64_t HW = (int64_t)a.W * a.H, HWt = (int64_t)a.Wt * a.Ht;
    const int u = blockIdx.x * SC_BX + threadIdx.x;
    const int v = blockIdx.y * SC_BY + threadIdx.y;
    if (u >= a.W || v >= a.H) return;
    const int k = blockIdx.z;
    const int src = v * a.W + u;
    const float d = load_depth(reinterpret_cast<const DT *>(a.depth) + (size_t)k * HW + src);
    const Geo g = contract(a.v[k], u, v, d, a.Wt, a.Ht, 1, a.max_hw);
    float gd = 0.0f;
    float3 gc = make_float3(0.0f, 0.0f, 0.0f);
    if (g.ok) {
        const float4 c = load_color(reinterpret_cast<const CT *>(a.color) + (size_t)k * HW + src);
        const float z = g.z;
        const float dx_dd = (g.m0 - g.x * g.m2) / z, dy_dd = (g.m1 - g.y * g.m2) / z;
        const float rho = a.v[k].f_ratio * (d / z);
        const float dhw_dd = (0.5f * rho > 0.5f && 0.5f * rho < a.max_hw)
                                 ? 0.5f * a.v[k].f_ratio * a.v[k].xf.b[2] / (z * z) : 0.0f;
        const float sig = 0.5f * g.hw, dsig_dd = 0.5f * dhw_dd;
        const float inv_s2 = 1.0f / (sig * sig);
        // d w / d d = w (-(ex dx/dd + ey dy/dd) / sig^2 + r^2 (dsig/dd) / sig^3)
        const float kr = dsig_dd * inv_s2 / sig;
        const int32_t *win = a.winner + (size_t)k * HWt;
        const float *wdep = a.warped_depth + (size_t)k * HWt;
        const float *wsum = a.wsum + (size_t)k * HWt;
        const float4 *oc = a.out_color + (size_t)k * HWt;
        for (int jj = g.j0; jj <= g.j1; ++jj)
            for (int ii = g.i0; ii <= g.i1; ++ii) {
                const size_t tp = (size_t)jj * a.Wt + ii;
                if (BLENDED) {
                    if (win[tp] == src) gd += a.grad_pixel[tp].w * g.m2;
                } else if (a.grad_depth && win[tp] == src) {
                    gd += a.grad_depth[(size_t)k * HWt + tp] * g.m2;
                }
                if (!(z <= __fadd_rn(wdep[tp], a.mu_band))) continue;
                const float ex = g.x - (float)ii, ey = g.y - (float)jj;
                const float r2 = ex * ex + ey * ey;
                const float w = expf(-0.5f * r2 * inv_s2);
                const float dw_dd = w * (-(ex * dx_dd + ey * dy_dd) * inv_s2 + r2 * kr);
                const float inv_sw = 1.0f / wsum[tp];
                const float4 G = BLENDED ? a.grad_pixel[tp] : a.grad_color[(size_t)k * HWt + tp];
                const float4 I = oc[tp];
                gc.x += G.x * w * inv_sw;
                gc.y += G.y * w * inv_sw;
                gc.z += G.z * w * inv_sw;
                gd += (G.x * (c.x - I.x) + G.y * (c.y - I.y) + G.z * (c.z - I.z)) * inv_sw * dw_dd;
            }
    }
    a.grad_in_depth[(size_t)k * HW + src] = gd;
    a.grad_in_color[(size_t)k * HW + src] = make_float4(gc.x, gc.y, gc.z, 0.0f);
}

template <typename DT, typename CT>
void soft_bwd_launch(const SplatArgs &a, dim3 grid, dim3 block, cudaStream_t st) {
    if (a.grad_pixel) soft_bwd<DT, CT, true><<<grid, block, 0, st>>>(a);
    else soft_bwd<DT, CT, false><<<grid, block, 0, st>>>(a);
}

template <typename DT, typename CT>
void soft_groups(const SplatArgs &a, int K, cudaStream_t st) {
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int slots = a.slots < K ? a.slots : K;
    for (int k0 = 0; k0 < K; k0 += slots) {
        const int kn = (K - k0) < slots ? (K - k0) : slots;
        splat_scatter<DT><<<scatter_grid(a.W, a.H, kn), dim3(SC_BX, SC_BY), 0, st>>>(a, k0);
        soft_accum<DT, CT><<<scatter_grid(a.W, a.H, kn), dim3(SC_BX, SC_BY), 0, st>>>(a, k0);
        if (tma_soft_resolve_ok(a, HWt))
            soft_resolve_tma<<<dim3((unsigned)((HWt + ST_PX - 1) / ST_PX), (unsigned)kn), 256, 0, st>>>(a, k0);
        else if (wide_soft_resolve_ok(a, HWt))
            soft_resolve_wide<<<dim3((unsigned)((HWt / 8 + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
        else if (HWt % 4 == 0)
            soft_resolve4<<<dim3((unsigned)((HWt / 4 + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
        else
            soft_resolve<<<dim3((unsigned)((HWt + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
    }
}

}  // namespace

cudaError_t launch_splat(const SplatArgs &a, int K, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
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
        const dim3 g = scatter_grid(a.W, a.H, kn), b(SC_BX, SC_BY);
        if (a.depth_dtype == GVS_F16) {
            if (a.guide_reject) splat_scatter<__half, true><<<g, b, 0, st>>>(a, k0);
            else splat_scatter<__half><<<g, b, 0, st>>>(a, k0);
        } else {
            if (a.guide_reject) splat_scatter<float, true><<<g, b, 0, st>>>(a, k0);
            else splat_scatter<float><<<g, b, 0, st>>>(a, k0);
        }
        if (tma_resolve_ok(a, HWt))
            splat_resolve_tma<<<dim3((unsigned)((HWt + RT_PX - 1) / RT_PX), (unsigned)kn), 256, 0, st>>>(a, k0);
        else if (HWt % 8 == 0)
            splat_resolveP<8><<<dim3((unsigned)((HWt / 8 + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
        else if (HWt % 4 == 0)
            splat_resolveP<4><<<dim3((unsigned)((HWt / 4 + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
        else
            splat_resolve<<<dim3((unsigned)((HWt + 255) / 256), (unsigned)kn), 256, 0, st>>>(a, k0);
    }
    return cudaGetLastError();
}

cudaError_t launch_soft_splat(const SplatArgs &a, int K, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const int64_t HWt = (int64_t)a.Wt * a.Ht;
    const int slots = a.slots < K ? a.slots : K;
    {
        const int64_t n = HWt * slots;
        int64_t blocks = (n / 2 + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        clear_keys<<<(unsigned)blocks, 256, 0, st>>>(a.keys, n);
        cudaError_t e = cudaMemsetAsync(a.acc, 0, (size_t)n * sizeof(float4), st);
        if (e != cudaSuccess) return e;
    }
    if (a.depth_dtype == GVS_F16) {
        if (a.color_dtype == GVS_BF16) soft_groups<__half, uint2>(a, K, st);
        else soft_groups<__half, float4>(a, K, st);
    } else {
        if (a.color_dtype == GVS_BF16) soft_groups<float, uint2>(a, K, st);
        else soft_groups<float, float4>(a, K, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_soft_splat_backward(const SplatArgs &a, int K, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const dim3 grid = scatter_grid(a.W, a.H, K), block(SC_BX, SC_BY);
    if (a.depth_dtype == GVS_F16) {
        if (a.color_dtype == GVS_BF16) soft_bwd_launch<__half, uint2>(a, grid, block, st);
        else soft_bwd_launch<__half, float4>(a, grid, block, st);
    } else {
        if (a.color_dtype == GVS_BF16) soft_bwd_launch<float, uint2>(a, grid, block, st);
        else soft_bwd_launch<float, float4>(a, grid, block, st);
    }
    return cudaGetLastError();
}

namespace {

// Supplement A.2: the target-view difference mask is the largest of the
// views' masks at their z-buffer winners (1 where no view covers the pixel),
// and w_tmp = min(beta_t (w_tmp_prev + w_view_prev) max(1 - M, 0), eta).
template <typename MK>
__global__ void __launch_bounds__(256) temporal_weight_kernel(const MK *__restrict__ masks, const int32_t *__restrict__ winner,
                                                              int K, int64_t HW, int64_t HWt,
                                                              const float *__restrict__ w_tmp_prev,
                                                              const float *__restrict__ w_view_prev, float beta_t,
                                                              float eta, float *__restrict__ w_tmp,
                                                              float *__restrict__ target_mask) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HWt) return;
    float M = -1.0f;
    for (int k = 0; k < K; ++k) {
        const int32_t w = winner[(size_t)k * HWt + p];
        if (w >= 0) M = fmaxf(M, (float)masks[(size_t)k * HW + w]);
    }
    if (M < 0.0f) M = 1.0f;
    if (target_mask) target_mask[p] = M;
    const float keep = fmaxf(1.0f - M, 0.0f);
    w_tmp[p] = fminf(beta_t * (w_tmp_prev[p] + w_view_prev[p]) * keep, eta);
}

// One row of blocks per view (gridDim.y = K).  V = 4: four pixels per thread with 16-byte
// depth and fused loads and 4-byte alpha and mask accesses (HWt a multiple of 4, planes
// aligned); V = 1: one pixel per thread.
template <int V>
__global__ void __launch_bounds__(256) guided_mask_kernel(const float *__restrict__ warped_depth,
                                                          const uint8_t *__restrict__ alpha,
                                                          const float *__restrict__ fused, int64_t HWt,
                                                          float mu_guide, uint8_t *__restrict__ guided) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t base = (size_t)blockIdx.y * HWt;
    if (V == 4) {
        if (4 * q >= HWt) return;
        const float4 d = __ldg(reinterpret_cast<const float4 *>(warped_depth + base) + q);
        const float4 f = __ldg(reinterpret_cast<const float4 *>(fused) + q);
        const uchar4 a = __ldg(reinterpret_cast<const uchar4 *>(alpha + base) + q);
        uchar4 g;
        g.x = (unsigned char)(a.x && fabsf(d.x - f.x) <= mu_guide);
        g.y = (unsigned char)(a.y && fabsf(d.y - f.y) <= mu_guide);
        g.z = (unsigned char)(a.z && fabsf(d.z - f.z) <= mu_guide);
        g.w = (unsigned char)(a.w && fabsf(d.w - f.w) <= mu_guide);
        reinterpret_cast<uchar4 *>(guided + base)[q] = g;
    } else {
        if (q >= HWt) return;
        guided[base + q] = (uint8_t)(alpha[base + q] && fabsf(warped_depth[base + q] - fused[q]) <= mu_guide);
    }
}

}  // namespace

cudaError_t launch_temporal_weight(const void *masks, int mask_dtype, const int32_t *winner, int K, int64_t HW,
                                   int64_t HWt, const float *w_tmp_prev, const float *w_view_prev, float beta_t,
                                   float eta, float *w_tmp, float *target_mask, cudaStream_t st) {
    const unsigned grid = (unsigned)((HWt + 255) / 256);
    if (mask_dtype == GVS_U8)
        temporal_weight_kernel<uint8_t><<<grid, 256, 0, st>>>(reinterpret_cast<const uint8_t *>(masks), winner, K,
                                                             HW, HWt, w_tmp_prev, w_view_prev, beta_t, eta, w_tmp,
                                                             target_mask);
    else
        temporal_weight_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float *>(masks), winner, K, HW,
                                                           HWt, w_tmp_prev, w_view_prev, beta_t, eta, w_tmp,
                                                           target_mask);
    return cudaGetLastError();
}

cudaError_t launch_guided_mask(const float *warped_depth, const uint8_t *alpha, const float *fused, int K,
                               int64_t HWt, float mu_guide, uint8_t *guided, cudaStream_t st) {
    if (K == 0 || HWt == 0) return cudaSuccess;
    if (HWt % 4 == 0 && aligned_to(warped_depth, 16) && aligned_to(fused, 16) && aligned_to(alpha, 4) &&
        aligned_to(guided, 4))
        guided_mask_kernel<4><<<dim3((unsigned)((HWt / 4 + 255) / 256), (unsigned)K), 256, 0, st>>>(
            warped_depth, alpha, fused, HWt, mu_guide, guided);
    else
        guided_mask_kernel<1><<<dim3((unsigned)((HWt + 255) / 256), (unsigned)K), 256, 0, st>>>(
            warped_depth, alpha, fused, HWt, mu_guide, guided);
    return cudaGetLastError();
}

GVS_BOUNDS_TAKE_FN(bounds_take_splat)

unsigned async_timeouts_take() {
    unsigned v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_async_timeouts, sizeof(v));
    cudaMemcpyToSymbol(g_async_timeouts, &z, sizeof(z));
    return v;
}

}  // namespace gvs
