// Device code shared by the fusion kernels (forward, batched, backward):
// map and depth loads, the nearest-pixel contract, the per-sample TSDF sum,
// the warp-bundle march with its slab tests, and the kernel-variant dispatch.
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "bounds_check.cuh"
#include "gvs_internal.cuh"

namespace gvs {
namespace {

#define kInf __int_as_float(0x7f800000)

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }

// Depth element load (FP32 or FP16) widened to FP32.
__device__ __forceinline__ float load_depth(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_depth(const __half *p) { return __half2float(__ldg(p)); }

// The depth as the map stores it: exact for float2, rounded to half for half2.
__device__ __forceinline__ float as_stored(float d, float2 *) { return d; }
__device__ __forceinline__ float as_stored(float d, __half2 *) { return __half2float(__float2half_rn(d)); }

__device__ __forceinline__ void store_map(float2 *p, float d, float w) { *p = make_float2(d, w); }
__device__ __forceinline__ void store_map(__half2 *p, float d, float w) { *p = __floats2half2_rn(d, w); }

__device__ __forceinline__ float2 load_map(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ float2 load_map(const __half2 *p) { return __half22float2(__ldg(p)); }

// Nearest integers (ties to even) of the exact real quotients hx/hz, hy/hz,
// hz > 0.  q = h * r with r = __fdividef(1, hz) (documented maximum error
// 2 ulp for 2^-126 <= hz <= 2^126) and one rounded product is within
// 3e-7 |q| of the quotient, so n = rint(q) is the answer whenever
// |q - n| + 4e-7 |q| <= 0.5.  Otherwise (rare: within a few 1e-4 pixel of a
// half-integer) the decision is re-taken from the signs of the exact
// residuals h - (n +/- 0.5) hz (one rounding each in the FMA, which never
// changes a sign).  The fix-up leaves n unchanged when q is not near a
// half-integer, so it runs for both coordinates under one branch.
__device__ __forceinline__ float exact_nearest_fixup(float num, float den, float n) {
    if (fabsf(n) < 4194304.0f) {
        const float hi = __fmaf_rn(-(n + 0.5f), den, num);
        const float lo = __fmaf_rn(-(n - 0.5f), den, num);
        const bool odd = (__float2int_rz(n) & 1) != 0;
        if (hi > 0.0f || (hi == 0.0f && odd)) n += 1.0f;
        else if (lo < 0.0f || (lo == 0.0f && odd)) n -= 1.0f;
    }
    return n;
}

// Nearest integer by the 1.5 * 2^23 shift: for |q| < 2^22 the sum q + 1.5 * 2^23
// lies in [2^23, 2^24), where the FP32 values are the integers, so the rounded
// sum is the shift plus rint(q) (ties to even: the shift is even) and its low
// bits hold rint(q) + 2^22.  Full-rate additions in place of a round and a
// conversion.
__device__ __forceinline__ float shift_round(float q, int &n) {
    const float t = __fadd_rn(q, 12582912.0f);
    n = __float_as_int(t) - 0x4B400000;
    return __fsub_rn(t, 12582912.0f);
}

// Every |q| >= 2^22 has a margin above 0.5 and takes the exact path; an
// infinite q (NaN margin) leaves a shifted index far outside any image, as the
// conversion would.
__device__ __forceinline__ void nearest_pixel(float hx, float hy, float hz, int &u, int &v) {
    const float r = __fdividef(1.0f, hz);
    const float qx = hx * r, qy = hy * r;
    int iu, iv;
    const float nx = shift_round(qx, iu), ny = shift_round(qy, iv);
    const float mx = fmaf(fabsf(qx), 4e-7f, fabsf(qx - nx));
    const float my = fmaf(fabsf(qy), 4e-7f, fabsf(qy - ny));
    if (fmaxf(mx, my) > 0.5f) {
        iu = __float2int_rz(exact_nearest_fixup(hx, hz, rintf(qx)));
        iv = __float2int_rz(exact_nearest_fixup(hy, hz, rintf(qy)));
    }
    u = iu;
    v = iv;
}

#ifndef GVS_FUSE_WARPS
#define GVS_FUSE_WARPS 4        // warps (bundles) per fusion block
#endif
constexpr int FZ_WARPS = GVS_FUSE_WARPS;
#ifndef GVS_FUSE_MIN_BLOCKS
#define GVS_FUSE_MIN_BLOCKS 9   // resident blocks per SM requested from the register allocator (56 registers)
#endif
constexpr int SKIP_COOL = 3;    // samples evaluated after both slab tests fail, before testing again

// Bundle shape and slab-test lengths of the march.  Every variant computes the
// same result; they differ only in speed, and the autotuner picks one per
// workload (gvs_fuse_params.variant).
//   bx x by : target pixels one warp marches together (bx * by = 32)
//   llong   : samples per segment in the first slab test
//   lshort  : samples per segment in the second test when the first fails
//   full    : the call has exactly KMAX views, so the per-view guard k < K
//             compiles away and the unrolled views form one block of code
//   spt     : samples each lane evaluates at once in a run of evaluations
//             (1 or 2: two keep twice the gathers in flight)
//   warp    : the mapping.  false: lane per ray (a bundle of bx x by = 32 rays per
//             warp); true: warp per ray (bx = by = 1), its lanes split into
//             views x samples, so a step evaluates 32 / KMAX consecutive samples
//             of the one ray at once and its slab tests hold for that ray alone
template <int BX_, int BY_, int LLONG_, int LSHORT_, bool FULL_ = false, int SPT_ = 1, bool WARP_ = false>
struct Tile {
    static constexpr int bx = BX_, by = BY_, llong = LLONG_, lshort = LSHORT_, spt = SPT_;
    static constexpr bool full = FULL_, warp = WARP_;
    static_assert(warp ? (bx == 1 && by == 1 && spt == 1) : bx * by == 32, "a bundle is one warp, or one ray");
    static_assert(llong >= 1 && lshort >= 1, "skip lengths must advance the march");
    static_assert(spt == 1 || spt == 2, "one or two samples at once");
};
template <typename T>
struct FullTile;
template <int BX_, int BY_, int LLONG_, int LSHORT_, bool FULL_, int SPT_, bool WARP_>
struct FullTile<Tile<BX_, BY_, LLONG_, LSHORT_, FULL_, SPT_, WARP_>> {
    using type = Tile<BX_, BY_, LLONG_, LSHORT_, true, SPT_, WARP_>;
};
using Tile0 = Tile<8, 4, 8, 2>;
using Tile1 = Tile<8, 4, 16, 4>;
using Tile2 = Tile<16, 2, 8, 2>;
using Tile3 = Tile<4, 8, 8, 2>;
using Tile4 = Tile<4, 8, 8, 2, false, 2>;
using Tile5 = Tile<8, 4, 8, 2, false, 2>;
using Tile6 = Tile<1, 1, 8, 2, false, 1, true>;
constexpr int kFuseVariants = 7;

struct Ray {
    float ax, ay, az;
};

// The bundle's rays between depths z0 and z1 fill a truncated pyramid (convex,
// 8 vertices: its 4 corner rays at z0 and z1).  In view k its points project
// inside the hull of the 8 vertex projections and their projected depths lie
// between the vertices' extremes (both statements exact for an affine depth
// and a projective map on a convex body in front of the camera; FP32 rounding
// of the samples is covered by a 1 pixel and 1e-6 relative margin).  A pixel
// of depth d can make a sample at projected depth z end a crossing only if
// d <= z (sdf <= 0) and d >= z - mu (not cut off), so the view is free over
// the slab when no valid depth in the pixel box around that hull lies in
// [zlo - 1.0001 mu, zhi] (every term positive or cut off), or the box is
// outside the image, or the slab is behind the camera.  One bound load: the
// finest tile level whose overlapping 2x2 block covers the box, else the whole
// view.  The bound's range decides first; failing that, its mask of occupied
// depth bins (a clear bin holds no depth; see DepthBound), which separates the
// surfaces of a tile that straddles a depth discontinuity.  When every view is free over the
// slab, no sample of it can end a crossing (S > 0 wherever W > 0).
// k is this lane's view; (b0, b1, b2) its offset b_k, held in registers so the
// lanes of a warp (testing different views) do not serialize on constant loads.
__device__ __forceinline__ bool slab_view_free(const FuseArgs &a, int k, const Ray (&corner)[4], float b0, float b1,
                                               float b2, float z0, float z1) {
    float xlo = kInf, xhi = -kInf, ylo = kInf, yhi = -kInf, zlo = kInf, zhi = -kInf;
    bool any_front = false, any_back = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float z = (c & 1) ? z1 : z0;
        const Ray &r = corner[c >> 1];
        const float hz = __fmaf_rn(z, r.az, b2);
        const float q = __fdividef(1.0f, hz);
        const float x = __fmaf_rn(z, r.ax, b0) * q;
        const float y = __fmaf_rn(z, r.ay, b1) * q;
        any_front |= hz > 1e-6f;
        any_back |= !(hz > 1e-6f);
        xlo = fminf(xlo, x); xhi = fmaxf(xhi, x);
        ylo = fminf(ylo, y); yhi = fmaxf(yhi, y);
        zlo = fminf(zlo, hz); zhi = fmaxf(zhi, hz);
    }
    zhi += 1e-6f * fabsf(zhi);
    zlo -= 1e-6f * fabsf(zlo);
    if (!any_front && zhi <= 1e-6f) return true;  // behind the camera throughout
    if (any_back) return false;                   // crosses the camera plane: do not try
    xlo -= 1.0f; xhi += 1.0f; ylo -= 1.0f; yhi += 1.0f;
    if (!(xlo <= xhi && ylo <= yhi)) return false;  // NaN
    if (xhi < 0.0f || yhi < 0.0f || xlo > (float)(a.W - 1) || ylo > (float)(a.H - 1)) return true;  // outside
    const int bx0 = min(max(__float2int_rd(xlo), 0), a.W - 1), bx1 = min(max(__float2int_ru(xhi), 0), a.W - 1);
    const int by0 = min(max(__float2int_rd(ylo), 0), a.H - 1), by1 = min(max(__float2int_ru(yhi), 0), a.H - 1);
    // a box spanning fewer than 2^l pixels per axis covers at most 2x2 tiles of level l
    const int span = max(bx1 - bx0, by1 - by0);
    const DepthBound *p;
    if (span < 16)
        p = a.ob[0] + ((size_t)k * a.th[0] + (by0 >> 4)) * a.tw[0] + (bx0 >> 4);
    else if (span < 32)
        p = a.ob[1] + ((size_t)k * a.th[1] + (by0 >> 5)) * a.tw[1] + (bx0 >> 5);
    else if (span < 64)
        p = a.ob[2] + ((size_t)k * a.th[2] + (by0 >> 6)) * a.tw[2] + (bx0 >> 6);
    else if (span < 128)
        p = a.ob[3] + ((size_t)k * a.th[3] + (by0 >> 7)) * a.tw[3] + (bx0 >> 7);
    else
        p = a.tg + k;
    if (!GVS_IN_BOUNDS(p - a.ob[0], (a.tg + a.K) - a.ob[0], GVS_SITE_FUSE_BOUNDS)) return false;
    const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p));
    const float lo = __uint_as_float(b.x), hi = __uint_as_float(b.y);
    const float qlo = __fsub_rn(zlo, a.behind);
    if (zhi < lo || qlo > hi) return true;
    // here lo <= zhi, so 0 <= m1, and m0 <= m1 (the bins are monotone)
    const int base = depth_bin(lo);
    const int m0 = min(max(depth_bin(fmaxf(qlo, 0.0f)) - base, 0), kDepthBins - 1);
    const int m1 = min(depth_bin(zhi) - base, kDepthBins - 1);
    const unsigned long long occupied = ((unsigned long long)b.w << 32) | b.z;
    return (occupied & (~0ull << m0) & (~0ull >> (kDepthBins - 1 - m1))) == 0ull;
}

// S and W of one sample over the input views (Supplement A.1), before the
// temporal term and the optional normalisation, exactly as the march computes them.
// A view whose sample lies behind its camera or off its image, or in front of
// the surface by more than mu, enters with weight 0 (a predicated gather, no
// branch): adding 0 * x leaves S and W as they were.
// FULL: the call has exactly KMAX views (no per-view guard).  PLANES: address
// view k's map through a.vb[k] (a constant-bank read for a __grid_constant__
// FuseArgs); otherwise from a.dw (where the arguments sit in global memory).
template <int KMAX, typename MT, bool FULL = false, bool PLANES = true>
__device__ __forceinline__ void evaluate_sample(const FuseArgs &a, const Ray (&ray)[KMAX], float zs, float &S,
                                                float &Wsum) {
    const size_t plane = (size_t)a.W * a.H;
    S = 0.0f;
    Wsum = 0.0f;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (FULL || k < a.K) {
            const float hz = __fmaf_rn(zs, ray[k].az, a.xf[k].b[2]);
            const float hx = __fmaf_rn(zs, ray[k].ax, a.xf[k].b[0]);
            const float hy = __fmaf_rn(zs, ray[k].ay, a.xf[k].b[1]);
            int u, v;
            nearest_pixel(hx, hy, hz, u, v);
            const bool in = hz > 1e-6f && (unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H &&
                            GVS_IN_BOUNDS((size_t)k * plane + (size_t)v * a.W + u, (size_t)a.K * plane,
                                          GVS_SITE_FUSE_MAP);
            float2 p = make_float2(0.0f, 0.0f);
            if (in) {
                const MT *plane_k = PLANES ? reinterpret_cast<const MT *>(a.vb[k])
                                           : reinterpret_cast<const MT *>(a.dw) + (size_t)k * plane;
                p = load_map(plane_k + (v * a.W + u));  // v W + u < 2^28
            }
            const float sdf = (p.x - hz) * a.inv_mu;
            const float w = (in && sdf >= -1.0f) ? p.y : 0.0f;
            S = fmaf(w, fminf(sdf, 1.0f), S);
            Wsum += w;
        }
    }
}

// Samples zs0 and zs1 at once (each exactly as evaluate_sample computes it): the
// two samples' gathers of a view are independent, so a lane keeps both in flight.
template <int KMAX, typename MT, bool FULL = false, bool PLANES = true>
__device__ __forceinline__ void evaluate_sample2(const FuseArgs &a, const Ray (&ray)[KMAX], float zs0, float zs1,
                                                 float &S0, float &W0, float &S1, float &W1) {
    const size_t plane = (size_t)a.W * a.H;
    S0 = W0 = S1 = W1 = 0.0f;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (FULL || k < a.K) {
            const MT *plane_k = PLANES ? reinterpret_cast<const MT *>(a.vb[k])
                                       : reinterpret_cast<const MT *>(a.dw) + (size_t)k * plane;
            float hz[2], pd[2], pw[2];
            bool in[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float zs = j ? zs1 : zs0;
                hz[j] = __fmaf_rn(zs, ray[k].az, a.xf[k].b[2]);
                const float hx = __fmaf_rn(zs, ray[k].ax, a.xf[k].b[0]);
                const float hy = __fmaf_rn(zs, ray[k].ay, a.xf[k].b[1]);
                int u, v;
                nearest_pixel(hx, hy, hz[j], u, v);
                in[j] = hz[j] > 1e-6f && (unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H &&
                        GVS_IN_BOUNDS((size_t)k * plane + (size_t)v * a.W + u, (size_t)a.K * plane,
                                      GVS_SITE_FUSE_MAP);
                float2 p = make_float2(0.0f, 0.0f);
                if (in[j]) p = load_map(plane_k + (v * a.W + u));
                pd[j] = p.x;
                pw[j] = p.y;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float sdf = (pd[j] - hz[j]) * a.inv_mu;
                const float w = (in[j] && sdf >= -1.0f) ? pw[j] : 0.0f;
                float &S = j ? S1 : S0;
                float &Wsum = j ? W1 : W0;
                S = fmaf(w, fminf(sdf, 1.0f), S);
                Wsum += w;
            }
        }
    }
}

// One warp per bundle of BX x BY target pixels.  The warp marches one sample
// index s for all its rays: cooperative slab tests (lane = view x segment,
// 32 / KMAX consecutive segments at once) skip runs of samples that hold no
// crossing end for any ray of the bundle; otherwise every ray still marching
// evaluates sample s (all KMAX views unrolled, one 8-byte gather each) and
// checks its own crossing.  The result equals the full uniform march.
// TMP: the temporal input (previous output depth and weight) and the views'
// weight at the crossing are compiled in only where they are used.  PLANES as
// in evaluate_sample.
template <int KMAX, typename MT, typename T, bool TMP = false, bool PLANES = true>
__device__ __forceinline__ void march_rays(const FuseArgs &a, int bundle, int lane) {
    constexpr int BX = T::bx, BY = T::by, SKIP_LONG = T::llong, SKIP_SHORT = T::lshort;
    constexpr int NSEG = 32 / KMAX;
    constexpr unsigned SEGMASK = KMAX == 32 ? 0xffffffffu : ((1u << KMAX) - 1u);
    const int nbx = (a.Wt + BX - 1) / BX;
    const int i0 = (bundle % nbx) * BX, j0 = (bundle / nbx) * BY;
    const int i1 = min(i0 + BX - 1, a.Wt - 1), j1 = min(j0 + BY - 1, a.Ht - 1);
    const int i = i0 + (lane % BX), j = j0 + (lane / BX);
    const bool inside = i < a.Wt && j < a.Ht;
    const float fi = (float)min(i, a.Wt - 1), fj = (float)min(j, a.Ht - 1);
    Ray ray[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (T::full || k < a.K) {
            const float *M = a.xf[k].M;
            ray[k].ax = __fmaf_rn(M[0], fi, __fmaf_rn(M[1], fj, M[2]));
            ray[k].ay = __fmaf_rn(M[3], fi, __fmaf_rn(M[4], fj, M[5]));
            ray[k].az = __fmaf_rn(M[6], fi, __fmaf_rn(M[7], fj, M[8]));
        }
    }
    // this lane's role in the slab tests: view tk of segment tseg
    const int tk = lane % KMAX, tseg = lane / KMAX;
    const bool tview = tk < a.K;
    Ray corner[4];
    float tb0, tb1, tb2;
    {
        const int kk = tview ? tk : 0;
        const float *M = a.xf[kk].M;
        tb0 = a.xf[kk].b[0];
        tb1 = a.xf[kk].b[1];
        tb2 = a.xf[kk].b[2];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float ci = (float)((c & 1) ? i1 : i0), cj = (float)((c & 2) ? j1 : j0);
            corner[c].ax = __fmaf_rn(M[0], ci, __fmaf_rn(M[1], cj, M[2]));
            corner[c].ay = __fmaf_rn(M[3], ci, __fmaf_rn(M[4], cj, M[5]));
            corner[c].az = __fmaf_rn(M[6], ci, __fmaf_rn(M[7], cj, M[8]));
        }
    }
    // temporal input at this ray's pixel, and its depth range over the bundle's rays
    float td = 0.0f, tw = 0.0f;
    if (TMP && a.tmp_depth && inside) {
        const size_t o = (size_t)j * a.Wt + i;
        const float d = a.tmp_depth[o], w = a.tmp_weight[o];
        if (valid_depth(d) && w > 0.0f) {
            td = d;
            tw = w;
        }
    }
    float tlo = tw > 0.0f ? td : kInf, thi = tw > 0.0f ? td : -kInf;
    if (TMP) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            tlo = fminf(tlo, __shfl_xor_sync(0xffffffffu, tlo, m));
            thi = fmaxf(thi, __shfl_xor_sync(0xffffffffu, thi, m));
        }
    }
    float S_prev = 0.0f, W_prev = 0.0f, z_prev = 0.0f, Wv_prev = 0.0f;
    float wview = 0.0f;
    bool have_prev = false;  // sample s-1 was evaluated (uniform across the warp)
    bool done = !inside;
    float out = 0.0f;
    int idx = -1;
    int s = 0;
    int cool = 0;
    bool shorter = false;
    while (s < a.D) {
        if (__all_sync(0xffffffffu, done)) break;
        if (cool == 0 && s < a.D - 1) {
            const int L = shorter ? SKIP_SHORT : SKIP_LONG;
            const int sa = s + tseg * L;
            bool f = false;
            if (sa < a.D - 1) {
                const int sb = min(sa + L, a.D - 1);
                const float z0 = __fmaf_rn((float)sa, a.dz, a.zn), z1 = __fmaf_rn((float)sb, a.dz, a.zn);
                f = !tview || slab_view_free(a, tk, corner, tb0, tb1, tb2, z0, z1);
                // the temporal input sits at the ray's own pixel: its projected depth is the sample depth
                if (TMP) f = f && (z1 < tlo || z0 > thi + a.behind);
            }
            const unsigned ball = __ballot_sync(0xffffffffu, f);
            int nfree = 0;
#pragma unroll
            for (int g = 0; g < NSEG; ++g) {
                if (nfree == g && ((ball >> (g * KMAX)) & SEGMASK) == SEGMASK) ++nfree;
            }
            if (nfree > 0) {
                s = min(s + nfree * L, a.D - 1);  // samples up to s are not crossing ends; s is evaluated next
                if (s == a.D - 1) break;           // ... unless it is the last: nothing follows it
                have_prev = false;
                shorter = false;
                continue;
            }
            if (!shorter && SKIP_SHORT < SKIP_LONG) {
                shorter = true;
                continue;
            }
            shorter = false;
            cool = SKIP_COOL;
        }
        // every lane evaluates (the warp issues the sample anyway); lanes still marching record it
        const int nev = (T::spt == 2 && cool >= 2 && s + 1 < a.D) ? 2 : 1;
        const float zs0 = __fmaf_rn((float)s, a.dz, a.zn);
        float Se[2], We[2], ze[2];
        ze[0] = zs0;
        if (T::spt == 2 && nev == 2) {
            ze[1] = __fmaf_rn((float)(s + 1), a.dz, a.zn);
            evaluate_sample2<KMAX, MT, T::full, PLANES>(a, ray, ze[0], ze[1], Se[0], We[0], Se[1], We[1]);
        } else {
            evaluate_sample<KMAX, MT, T::full, PLANES>(a, ray, zs0, Se[0], We[0]);
        }
#pragma unroll
        for (int e = 0; e < T::spt; ++e) {
            if (e < nev) {
                const float zs = ze[e];
                float S = Se[e], Wsum = We[e];
                if (!done) {
                    const float Wv = Wsum;
                    if (TMP && tw > 0.0f) {
                        const float sdf = (td - zs) * a.inv_mu;
                        if (sdf >= -1.0f) {
                            S = fmaf(tw, fminf(sdf, 1.0f), S);
                            Wsum += tw;
                        }
                    }
                    if (a.normalize && Wsum > 0.0f) S = S / Wsum;
                    if (have_prev && W_prev > 0.0f && Wsum > 0.0f && S_prev > 0.0f && S <= 0.0f) {
                        const float t = S_prev / (S_prev - S);
                        out = z_prev + (zs - z_prev) * t;
                        if (TMP) wview = Wv_prev + t * (Wv - Wv_prev);
                        idx = s - 1;
                        done = true;
                    }
                    S_prev = S;
                    W_prev = Wsum;
                    Wv_prev = Wv;
                    z_prev = zs;
                }
                have_prev = true;
                ++s;
                if (cool > 0) --cool;
            }
        }
    }
    if (inside) {
        const size_t o = (size_t)j * a.Wt + i;
        a.fused[o] = out;
        if (a.crossing) a.crossing[o] = (int16_t)idx;
        if (TMP && a.wview) a.wview[o] = wview;
    }
}

// One warp per target ray (the warp-per-pixel mapping; `pixel` < Wt * Ht).  Lane
// (q, k) = (lane / KMAX, lane % KMAX) takes view k: in a slab test, segment q of
// the ray's own slab (its four corner rays are the ray itself); in a run of
// evaluations, sample s + q.  Each sample's S and W are summed over the views in
// view order from the lanes' terms, exactly as evaluate_sample sums them, and the
// samples are then scanned in order, so the crossing, its index and its depth are
// bit for bit those of march_rays (and of the full uniform march).  No temporal
// input.
template <int KMAX, typename MT, typename T, bool PLANES = true>
__device__ __forceinline__ void march_ray_warp(const FuseArgs &a, int pixel, int lane) {
    constexpr int NQ = 32 / KMAX;  // samples per step = segments per slab test
    constexpr unsigned SEGMASK = KMAX == 32 ? 0xffffffffu : ((1u << KMAX) - 1u);
    constexpr int SKIP_LONG = T::llong, SKIP_SHORT = T::lshort;
    const int i = pixel % a.Wt, j = pixel / a.Wt;
    const float fi = (float)i, fj = (float)j;
    const int tk = lane % KMAX, tq = lane / KMAX;
    const bool tview = T::full || tk < a.K;
    const int kk = tview ? tk : 0;
    const size_t plane = (size_t)a.W * a.H;
    Ray corner[4];
    float tb0, tb1, tb2;
    {
        const float *M = a.xf[kk].M;
        tb0 = a.xf[kk].b[0];
        tb1 = a.xf[kk].b[1];
        tb2 = a.xf[kk].b[2];
        corner[0].ax = __fmaf_rn(M[0], fi, __fmaf_rn(M[1], fj, M[2]));
        corner[0].ay = __fmaf_rn(M[3], fi, __fmaf_rn(M[4], fj, M[5]));
        corner[0].az = __fmaf_rn(M[6], fi, __fmaf_rn(M[7], fj, M[8]));
        corner[1] = corner[2] = corner[3] = corner[0];
    }
    const Ray &ray = corner[0];
    const MT *plane_k = PLANES ? reinterpret_cast<const MT *>(a.vb[kk])
                               : reinterpret_cast<const MT *>(a.dw) + (size_t)kk * plane;
    float S_prev = 0.0f, W_prev = 0.0f, z_prev = 0.0f;
    bool have_prev = false;
    float out = 0.0f;
    int idx = -1;
    int s = 0, cool = 0;
    bool shorter = false;
    while (s < a.D) {
        if (cool == 0 && s < a.D - 1) {
            const int L = shorter ? SKIP_SHORT : SKIP_LONG;
            const int sa = s + tq * L;
            bool f = false;
            if (sa < a.D - 1) {
                const int sb = min(sa + L, a.D - 1);
                const float z0 = __fmaf_rn((float)sa, a.dz, a.zn), z1 = __fmaf_rn((float)sb, a.dz, a.zn);
                f = !tview || slab_view_free(a, tk, corner, tb0, tb1, tb2, z0, z1);
            }
            const unsigned ball = __ballot_sync(0xffffffffu, f);
            int nfree = 0;
#pragma unroll
            for (int g = 0; g < NQ; ++g) {
                if (nfree == g && ((ball >> (g * KMAX)) & SEGMASK) == SEGMASK) ++nfree;
            }
            if (nfree > 0) {
                s = min(s + nfree * L, a.D - 1);
                if (s == a.D - 1) break;
                have_prev = false;
                shorter = false;
                continue;
            }
            if (!shorter && SKIP_SHORT < SKIP_LONG) {
                shorter = true;
                continue;
            }
            shorter = false;
            cool = SKIP_COOL;
        }
        // this lane's term of sample s + tq in view tk, as evaluate_sample forms it
        float w = 0.0f, t = 0.0f;
        if (s + tq < a.D && tview) {
            const float zs = __fmaf_rn((float)(s + tq), a.dz, a.zn);
            const float hz = __fmaf_rn(zs, ray.az, tb2);
            const float hx = __fmaf_rn(zs, ray.ax, tb0);
            const float hy = __fmaf_rn(zs, ray.ay, tb1);
            int u, v;
            nearest_pixel(hx, hy, hz, u, v);
            const bool in = hz > 1e-6f && (unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H &&
                            GVS_IN_BOUNDS((size_t)kk * plane + (size_t)v * a.W + u, (size_t)a.K * plane,
                                          GVS_SITE_FUSE_MAP);
            float2 p = make_float2(0.0f, 0.0f);
            if (in) p = load_map(plane_k + (v * a.W + u));  // v W + u < 2^28
            const float sdf = (p.x - hz) * a.inv_mu;
            w = (in && sdf >= -1.0f) ? p.y : 0.0f;
            t = fminf(sdf, 1.0f);
        }
        // S and W of sample s + tq: its group's terms in view order
        float S = 0.0f, Wsum = 0.0f;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const float wk = __shfl_sync(0xffffffffu, w, tq * KMAX + k);
            const float tk_ = __shfl_sync(0xffffffffu, t, tq * KMAX + k);
            if (T::full || k < a.K) {
                S = fmaf(wk, tk_, S);
                Wsum += wk;
            }
        }
        // the step's samples in order
        bool done = false;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float Sq = __shfl_sync(0xffffffffu, S, q * KMAX);
            const float Wq = __shfl_sync(0xffffffffu, Wsum, q * KMAX);
            if (!done && s < a.D) {
                const float zs = __fmaf_rn((float)s, a.dz, a.zn);
                if (a.normalize && Wq > 0.0f) Sq = Sq / Wq;
                if (have_prev && W_prev > 0.0f && Wq > 0.0f && S_prev > 0.0f && Sq <= 0.0f) {
                    const float tt = S_prev / (S_prev - Sq);
                    out = z_prev + (zs - z_prev) * tt;
                    idx = s - 1;
                    done = true;
                }
                S_prev = Sq;
                W_prev = Wq;
                z_prev = zs;
                have_prev = true;
                ++s;
                if (cool > 0) --cool;
            }
        }
        if (done) break;
    }
    if (lane == 0) {
        const size_t o = (size_t)j * a.Wt + i;
        a.fused[o] = out;
        if (a.crossing) a.crossing[o] = (int16_t)idx;
    }
}

template <int KMAX, typename MT, typename T, bool TMP = false, bool PLANES = true>
__device__ __forceinline__ void march_bundle(const FuseArgs &a, int bundle, int lane) {
    if constexpr (T::warp) {
        static_assert(!TMP, "the warp-per-ray march takes no temporal input");
        march_ray_warp<KMAX, MT, T, PLANES>(a, bundle, lane);
    } else {
        march_rays<KMAX, MT, T, TMP, PLANES>(a, bundle, lane);
    }
}

// Calls F<Tile_i>::run(...) for the variant, with the full form of the tile
// when the call has exactly KMAX views; views counts other than 8 and 16 use
// the default tile only (fewer instantiations to build), except the
// warp-per-ray variant 6, built for 8, 16 and 32 views (5 to 32 views).
template <int KMAX, typename MT, template <int, typename, typename> class F, typename T, typename... Args>
void full_or_not(int K, Args... args) {
    if (K == KMAX) F<KMAX, MT, typename FullTile<T>::type>::run(args...);
    else F<KMAX, MT, T>::run(args...);
}

template <int KMAX, typename MT, template <int, typename, typename> class F, typename... Args>
void by_variant(int K, int variant, Args... args) {
    if constexpr (KMAX >= 8) {  // the warp-per-ray mapping: 8, 16 and 32-view kernels
        if (variant == 6) {
            full_or_not<KMAX, MT, F, Tile6>(K, args...);
            return;
        }
    }
    if (KMAX == 8 || KMAX == 16) {
        switch (variant) {
            case 1: full_or_not<KMAX, MT, F, Tile1>(K, args...); return;
            case 2: full_or_not<KMAX, MT, F, Tile2>(K, args...); return;
            case 3: full_or_not<KMAX, MT, F, Tile3>(K, args...); return;
            case 4: full_or_not<KMAX, MT, F, Tile4>(K, args...); return;
            case 5: full_or_not<KMAX, MT, F, Tile5>(K, args...); return;
            default: break;
        }
    }
    full_or_not<KMAX, MT, F, Tile0>(K, args...);
}

template <template <int, typename, typename> class F, typename... Args>
void by_kmax(int K, int map_dtype, int variant, Args... args) {
    if (map_dtype == GVS_F16) {
        if (K <= 4) by_variant<4, __half2, F>(K, variant, args...);
        else if (K <= 8) by_variant<8, __half2, F>(K, variant, args...);
        else if (K <= 16) by_variant<16, __half2, F>(K, variant, args...);
        else by_variant<32, __half2, F>(K, variant, args...);
    } else {
        if (K <= 4) by_variant<4, float2, F>(K, variant, args...);
        else if (K <= 8) by_variant<8, float2, F>(K, variant, args...);
        else if (K <= 16) by_variant<16, float2, F>(K, variant, args...);
        else by_variant<32, float2, F>(K, variant, args...);
    }
}

// The same for kernels built with the default tile only.
template <template <int, typename, typename> class F, typename... Args>
void by_kmax_tile0(int K, int map_dtype, Args... args) {
    if (map_dtype == GVS_F16) {
        if (K <= 4) full_or_not<4, __half2, F, Tile0>(K, args...);
        else if (K <= 8) full_or_not<8, __half2, F, Tile0>(K, args...);
        else if (K <= 16) full_or_not<16, __half2, F, Tile0>(K, args...);
        else full_or_not<32, __half2, F, Tile0>(K, args...);
    } else {
        if (K <= 4) full_or_not<4, float2, F, Tile0>(K, args...);
        else if (K <= 8) full_or_not<8, float2, F, Tile0>(K, args...);
        else if (K <= 16) full_or_not<16, float2, F, Tile0>(K, args...);
        else full_or_not<32, float2, F, Tile0>(K, args...);
    }
}

}  // namespace
}  // namespace gvs
