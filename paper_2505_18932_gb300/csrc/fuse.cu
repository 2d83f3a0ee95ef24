// Image-based TSDF fusion in the target view (Supplement A.1, Eq. 3).
//
// weight_map  : the confidence weight of Supplement A.1 depends only on the
//               sampled input pixel (nearest-pixel sampling), so it is
//               computed once per input pixel and packed with the depth as
//               float2 (d, omega); an invalid pixel is stored as (0, 0), whose
//               signed distance is below -1 so it never contributes.  7x7
//               stencil over a shared-memory tile with halo.  The same kernel
//               writes the min/max valid depth of every 8x8 tile.
// depth_bounds, bounds_overlap: build the per-view bound pyramid (8, 32 and
//               128 pixel tiles, each also as overlapping 2x2-tile blocks, and
//               the whole view) from the 8x8 tiles.
// fuse        : one warp per 8x4 bundle of target pixels, one thread per ray,
//               marching the D samples in registers (one 8-byte gather per
//               sample and view) to the first +/- crossing.  Before evaluating
//               samples the warp tries to prove that a run of them holds no
//               crossing end for any ray of the bundle (see slab_view_free);
//               such runs are skipped.  A skipped sample provably has S > 0 or
//               W = 0, so the first crossing, its index and its interpolated
//               depth are exactly those of the full uniform march.
#include <cuda_fp16.h>
#include <math.h>

#include "gvs_internal.cuh"

namespace gvs {
namespace {

constexpr int WM_TX = 32;   // block of 32 x 32 output pixels: 32 x 8 threads,
constexpr int WM_TY = 32;   // each thread a column of WM_P pixels
constexpr int WM_P = 4;
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

// R = window / 2.  The shared tile holds the block's depths, as the map will
// store them, plus an R-pixel halo replicated at the image borders (invalid
// depths as NaN).  A thread reads each of the (WM_P + 2R) x (2R + 1) shared
// values its column needs once and reuses it for every output whose window
// contains it.  DT: float or __half input; MT: float2 or __half2 map.
template <int R, typename DT, typename MT>
__global__ void __launch_bounds__(256) weight_map_kernel(const DT *__restrict__ depth, char *__restrict__ map,
                                                         MapLayout L, float mu, float wconst, float inv_w2) {
    constexpr int SW = WM_TX + 2 * R;
    constexpr int SH = WM_TY + 2 * R;
    __shared__ float tile[SH][SW];
    __shared__ float2 red[WM_TY / WM_P][WM_TX / 8];
    const int W = L.W, H = L.H;
    const int k = blockIdx.z;
    const DT *dep = depth + (size_t)k * W * H;
    const int x0 = blockIdx.x * WM_TX - R;
    const int y0 = blockIdx.y * WM_TY - R;
    const int tid = threadIdx.y * WM_TX + threadIdx.x;
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        // whole-view bounds, reduced into by depth_bounds with integer atomics on the float bits
        reinterpret_cast<int2 *>(map + L.off_g)[k] = make_int2(0x7f800000, (int)0xff800000u);
    }
    for (int e = tid; e < SW * SH; e += 256) {
        const int sy = e / SW, sx = e - sy * SW;
        const int gx = min(max(x0 + sx, 0), W - 1);
        const int gy = min(max(y0 + sy, 0), H - 1);
        const float d = as_stored(load_depth(&dep[(size_t)gy * W + gx]), (MT *)nullptr);
        tile[sy][sx] = valid_depth(d) ? d : __int_as_float(0x7fc00000);  // NaN marks invalid
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = blockIdx.x * WM_TX + tx;
    const int yb = blockIdx.y * WM_TY + ty * WM_P;
    float dc[WM_P], nu[WM_P];
#pragma unroll
    for (int p = 0; p < WM_P; ++p) {
        dc[p] = tile[ty * WM_P + p + R][tx + R];
        nu[p] = 0.0f;
    }
#pragma unroll
    for (int r = 0; r < WM_P + 2 * R; ++r) {
        float row[2 * R + 1];
#pragma unroll
        for (int dx = 0; dx <= 2 * R; ++dx) row[dx] = tile[ty * WM_P + r][tx + dx];
#pragma unroll
        for (int p = 0; p < WM_P; ++p) {
            if (r - p >= 0 && r - p <= 2 * R) {
#pragma unroll
                for (int dx = 0; dx <= 2 * R; ++dx) {
                    // fminf returns mu for a NaN (invalid) neighbour: it counts mu^2
                    const float t = fminf(fabsf(dc[p] - row[dx]), mu);
                    nu[p] = fmaf(t, t, nu[p]);
                }
            }
        }
    }
    float lo = kInf, hi = -kInf;
    MT *dw = reinterpret_cast<MT *>(map + L.off_dw) + (size_t)k * W * H;
#pragma unroll
    for (int p = 0; p < WM_P; ++p) {
        const int y = yb + p;
        if (x < W && y < H) {
            float d = 0.0f, w = 0.0f;
            if (dc[p] == dc[p]) {  // valid centre
                w = nu[p] > 0.0f ? fminf(wconst * rsqrtf(nu[p] * inv_w2), 1.0f) : 1.0f;
                d = dc[p];
                lo = fminf(lo, d);
                hi = fmaxf(hi, d);
            }
            store_map(&dw[(size_t)y * W + x], d, w);
        }
    }
    // 8x8 tile bounds: over the 8 lanes of a tile column group, then the two thread rows of a tile
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, m));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, m));
    }
    if ((tx & 7) == 0) red[ty][tx >> 3] = make_float2(lo, hi);
    __syncthreads();
    if (tid < (WM_TY / 8) * (WM_TX / 8)) {
        const int tc = tid % (WM_TX / 8), tr = tid / (WM_TX / 8);
        const float2 a = red[2 * tr][tc], b = red[2 * tr + 1][tc];
        const int gx = blockIdx.x * (WM_TX / 8) + tc, gy = blockIdx.y * (WM_TY / 8) + tr;
        if (gx < L.tw[0] && gy < L.th[0])
            reinterpret_cast<float2 *>(map + L.off_T[0])[((size_t)k * L.th[0] + gy) * L.tw[0] + gx] =
                make_float2(fminf(a.x, b.x), fmaxf(a.y, b.y));
    }
}

__device__ __forceinline__ float2 merge(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fmaxf(a.y, b.y)); }

// One block per (128x128 pixel tile, view), one thread per 8x8 tile: writes
// O_3 (needs one tile of halo right and below), T_5, T_7 and the view bounds.
__global__ void __launch_bounds__(256) depth_bounds_kernel(char *__restrict__ map, MapLayout L) {
    __shared__ float2 s[17][17];
    const int k = blockIdx.z;
    const float2 *T3 = reinterpret_cast<const float2 *>(map + L.off_T[0]) + (size_t)k * L.tw[0] * L.th[0];
    const int tid = threadIdx.y * 16 + threadIdx.x;
    for (int e = tid; e < 17 * 17; e += 256) {
        const int ly = e / 17, lx = e - ly * 17;
        const int tx = blockIdx.x * 16 + lx, ty = blockIdx.y * 16 + ly;
        s[ly][lx] = (tx < L.tw[0] && ty < L.th[0]) ? T3[(size_t)ty * L.tw[0] + tx] : make_float2(kInf, -kInf);
    }
    __syncthreads();
    const int x = threadIdx.x, y = threadIdx.y;
    const int tx = blockIdx.x * 16 + x, ty = blockIdx.y * 16 + y;
    if (tx < L.tw[0] && ty < L.th[0]) {
        const float2 o = merge(merge(s[y][x], s[y][x + 1]), merge(s[y + 1][x], s[y + 1][x + 1]));
        reinterpret_cast<float2 *>(map + L.off_O[0])[((size_t)k * L.th[0] + ty) * L.tw[0] + tx] = o;
    }
    if ((x & 3) == 0 && (y & 3) == 0) {
        float2 c = make_float2(kInf, -kInf);
#pragma unroll
        for (int dy = 0; dy < 4; ++dy)
#pragma unroll
            for (int dx = 0; dx < 4; ++dx) c = merge(c, s[y + dy][x + dx]);
        const int x5 = blockIdx.x * 4 + (x >> 2), y5 = blockIdx.y * 4 + (y >> 2);
        if (x5 < L.tw[1] && y5 < L.th[1])
            reinterpret_cast<float2 *>(map + L.off_T[1])[((size_t)k * L.th[1] + y5) * L.tw[1] + x5] = c;
    }
    if (tid == 0) {
        float2 c = make_float2(kInf, -kInf);
        for (int i = 0; i < 256; ++i) c = merge(c, s[i >> 4][i & 15]);
        reinterpret_cast<float2 *>(map + L.off_T[2])[((size_t)k * L.th[2] + blockIdx.y) * L.tw[2] + blockIdx.x] = c;
        int *g = reinterpret_cast<int *>(map + L.off_g) + 2 * k;
        if (c.x <= c.y) {  // the tile holds a valid depth
            atomicMin(&g[0], __float_as_int(c.x));  // positive floats order like their bits
            atomicMax(&g[1], __float_as_int(c.y));
        }
    }
}

// O_l from T_l for levels 5 and 7: one thread per (view, tile).
__global__ void __launch_bounds__(256) bounds_overlap_kernel(char *__restrict__ map, MapLayout L) {
    const int64_t n5 = (int64_t)L.tw[1] * L.th[1], n7 = (int64_t)L.tw[2] * L.th[2];
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)L.K * (n5 + n7)) return;
    const int k = (int)(q / (n5 + n7));
    q -= (int64_t)k * (n5 + n7);
    const int l = q < n5 ? 1 : 2;
    if (l == 2) q -= n5;
    const int tw = L.tw[l], th = L.th[l];
    const int tx = (int)(q % tw), ty = (int)(q / tw);
    const float2 *T = reinterpret_cast<const float2 *>(map + L.off_T[l]) + (size_t)k * tw * th;
    float2 o = T[(size_t)ty * tw + tx];
    if (tx + 1 < tw) o = merge(o, T[(size_t)ty * tw + tx + 1]);
    if (ty + 1 < th) o = merge(o, T[(size_t)(ty + 1) * tw + tx]);
    if (tx + 1 < tw && ty + 1 < th) o = merge(o, T[(size_t)(ty + 1) * tw + tx + 1]);
    reinterpret_cast<float2 *>(map + L.off_O[l])[((size_t)k * th + ty) * tw + tx] = o;
}

// Nearest integers (ties to even) of the exact real quotients hx/hz, hy/hz,
// hz > 0.  q = h * r with r ~ 1/hz (relative error a few ulp) is within 0.01
// of the quotient for any quotient that can land inside an image
// (|q| < 2^14 + 1); only when a q sits within 0.01 of a half-integer is the
// decision re-taken from the signs of the exact residuals h - (n +/- 0.5) hz
// (one rounding each in the FMA, which never changes a sign).  The fix-up
// leaves n unchanged when q is not near a half-integer, so it runs for both
// coordinates under one branch.
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

__device__ __forceinline__ void nearest_pixel(float hx, float hy, float hz, int &u, int &v) {
    const float r = __fdividef(1.0f, hz);
    const float qx = hx * r, qy = hy * r;
    float nx = rintf(qx), ny = rintf(qy);
    if (fmaxf(fabsf(qx - nx), fabsf(qy - ny)) > 0.49f) {
        nx = exact_nearest_fixup(hx, hz, nx);
        ny = exact_nearest_fixup(hy, hz, ny);
    }
    u = __float2int_rz(nx);
    v = __float2int_rz(ny);
}

constexpr int BX = 8;   // a warp marches a bundle of BX x BY target pixels
constexpr int BY = 4;
constexpr int FZ_WARPS = 4;
#ifndef GVS_FUSE_MIN_BLOCKS
#define GVS_FUSE_MIN_BLOCKS 8   // resident blocks per SM requested from the register allocator (64 registers)
#endif
#ifndef GVS_SKIP_LONG
#define GVS_SKIP_LONG 8    // samples per segment in the first test
#endif
#ifndef GVS_SKIP_SHORT
#define GVS_SKIP_SHORT 2   // samples per segment in the second test when the first fails
#endif
#ifndef GVS_SKIP_COOL
#define GVS_SKIP_COOL 4    // samples evaluated after both tests fail, before testing again
#endif
constexpr int SKIP_LONG = GVS_SKIP_LONG;
constexpr int SKIP_SHORT = GVS_SKIP_SHORT;
constexpr int SKIP_COOL = GVS_SKIP_COOL;
static_assert(SKIP_LONG >= 1 && SKIP_SHORT >= 1 && SKIP_COOL >= 0, "skip lengths must advance the march");

struct Ray {
    float ax, ay, az;
};

// The bundle's rays between depths z0 and z1 fill a truncated pyramid (convex,
// 8 vertices: its 4 corner rays at z0 and z1).  In view k its points project
// inside the hull of the 8 vertex projections and their projected depths lie
// between the vertices' extremes (both statements exact for an affine depth
// and a projective map on a convex body in front of the camera; FP32 rounding
// of the samples is covered by a 1 pixel and 1e-6 relative margin).  The view
// is free over the slab when every valid depth in the pixel box around that
// hull is strictly beyond the largest projected depth (sdf > 0: a positive
// term) or at least 1.0001 mu in front of the smallest (sdf < -1: cut off), or
// the box is outside the image, or the slab is behind the camera.  One bounds
// load: the finest tile level whose overlapping 2x2 block covers the box, else
// the whole view.  When every view is free over the slab, no sample of it can
// end a crossing (S > 0 wherever W > 0).
__device__ __forceinline__ bool slab_view_free(const FuseArgs &a, int k, const Ray (&corner)[4], float z0,
                                               float z1) {
    const float b0 = a.xf[k].b[0], b1 = a.xf[k].b[1], b2 = a.xf[k].b[2];
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
    const float2 *p;
    if (span < 8)
        p = a.ob[0] + ((size_t)k * a.th[0] + (by0 >> 3)) * a.tw[0] + (bx0 >> 3);
    else if (span < 32)
        p = a.ob[1] + ((size_t)k * a.th[1] + (by0 >> 5)) * a.tw[1] + (bx0 >> 5);
    else if (span < 128)
        p = a.ob[2] + ((size_t)k * a.th[2] + (by0 >> 7)) * a.tw[2] + (bx0 >> 7);
    else
        p = a.tg + k;
    const float2 b = __ldg(p);
    return zhi < b.x || zlo > b.y + a.behind;
}

// S and W of one sample (Supplement A.1), exactly as the full march computes them.
template <int KMAX, typename MT>
__device__ __forceinline__ void evaluate_sample(const FuseArgs &a, const Ray (&ray)[KMAX], float zs, float &S,
                                                float &Wsum) {
    const MT *map = reinterpret_cast<const MT *>(a.dw);
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
                if ((unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H) {
                    const float2 p = load_map(&map[(size_t)k * plane + (size_t)v * a.W + u]);
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
}

// One warp per bundle of BX x BY target pixels.  The warp marches one sample
// index s for all its rays: cooperative slab tests (lane = view x segment,
// 32 / KMAX consecutive segments at once) skip runs of samples that hold no
// crossing end for any ray of the bundle; otherwise every ray still marching
// evaluates sample s (all KMAX views unrolled, one 8-byte gather each) and
// checks its own crossing.  The result equals the full uniform march.
template <int KMAX, typename MT>
__global__ void __launch_bounds__(32 * FZ_WARPS, GVS_FUSE_MIN_BLOCKS) fuse_kernel(const FuseArgs a) {
    constexpr int NSEG = 32 / KMAX;
    constexpr unsigned SEGMASK = KMAX == 32 ? 0xffffffffu : ((1u << KMAX) - 1u);
    const int lane = threadIdx.x & 31;
    const int nbx = (a.Wt + BX - 1) / BX;
    const int nbundles = nbx * ((a.Ht + BY - 1) / BY);
    const int bundle = blockIdx.x * FZ_WARPS + (threadIdx.x >> 5);
    if (bundle >= nbundles) return;  // the whole warp leaves together
    const int i0 = (bundle % nbx) * BX, j0 = (bundle / nbx) * BY;
    const int i1 = min(i0 + BX - 1, a.Wt - 1), j1 = min(j0 + BY - 1, a.Ht - 1);
    const int i = i0 + (lane % BX), j = j0 + (lane / BX);
    const bool inside = i < a.Wt && j < a.Ht;
    const float fi = (float)min(i, a.Wt - 1), fj = (float)min(j, a.Ht - 1);
    Ray ray[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < a.K) {
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
    {
        const int kk = tview ? tk : 0;
        const float *M = a.xf[kk].M;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float ci = (float)((c & 1) ? i1 : i0), cj = (float)((c & 2) ? j1 : j0);
            corner[c].ax = __fmaf_rn(M[0], ci, __fmaf_rn(M[1], cj, M[2]));
            corner[c].ay = __fmaf_rn(M[3], ci, __fmaf_rn(M[4], cj, M[5]));
            corner[c].az = __fmaf_rn(M[6], ci, __fmaf_rn(M[7], cj, M[8]));
        }
    }
    float S_prev = 0.0f, W_prev = 0.0f, z_prev = 0.0f;
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
                f = !tview || slab_view_free(a, tk, corner, __fmaf_rn((float)sa, a.dz, a.zn),
                                             __fmaf_rn((float)sb, a.dz, a.zn));
            }
            const unsigned ball = __ballot_sync(0xffffffffu, f);
            int nfree = 0;
#pragma unroll
            for (int g = 0; g < NSEG; ++g) {
                if (nfree == g && ((ball >> (g * KMAX)) & SEGMASK) == SEGMASK) ++nfree;
            }
            if (nfree > 0) {
                s = min(s + nfree * L, a.D - 1);  // samples up to s are not crossing ends; s is evaluated next
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
        const float zs = __fmaf_rn((float)s, a.dz, a.zn);
        if (!done) {
            float S, Wsum;
            evaluate_sample<KMAX, MT>(a, ray, zs, S, Wsum);
            if (have_prev && W_prev > 0.0f && Wsum > 0.0f && S_prev > 0.0f && S <= 0.0f) {
                out = z_prev + (zs - z_prev) * (S_prev / (S_prev - S));
                idx = s - 1;
                done = true;
            }
            S_prev = S;
            W_prev = Wsum;
            z_prev = zs;
        }
        have_prev = true;
        ++s;
        if (cool > 0) --cool;
    }
    if (inside) {
        const size_t o = (size_t)j * a.Wt + i;
        a.fused[o] = out;
        if (a.crossing) a.crossing[o] = (int16_t)idx;
    }
}

// ---------------------------------------------------------------------------
// Adjoint of the fused depth (normalize = 0), in two passes.
//
// D = z_s + dz S_s / (S_s - S_{s+1}) depends on the inputs only through the
// two bracketing samples.  For a view contributing at one of them with
// clamped distance c, weight omega and signed distance sdf at input pixel q:
//   dD/dd(q) += g_S omega [-1 < sdf < 1] / mu                 (the clamp)
//   dD/dd(n) += g_S c domega(q)/dd(n)   for q's window entries n (the weight)
// with g_S = dD/dS of that sample.  The weight's derivative is linear in
// g_S c, so pass 1 (one thread per target pixel) accumulates, per sampled
// input pixel q, A(q) = sum g_S c and B(q) = sum g_S omega [...] / mu with one
// float2 atomic per (sample, view); pass 2 (one thread per input pixel x)
// applies domega/dnu and the window:
//   grad(x) = B(x) + P(x) sum_{entries n of x} 2 (d_x - d_n) [|d_x - d_n| < mu]
//           + sum_{c whose window holds x, with multiplicity}
//                 P(c) (-2) (d_c - d_x) [|d_c - d_x| < mu]
// where P(c) = A(c) domega/dnu(c) (0 when the weight is saturated or c is
// invalid).  Nothing of size D x H x W is stored; the bracketing samples are
// recomputed by the forward's own code, so they are bit-identical to it.
// ---------------------------------------------------------------------------

template <int KMAX, typename MT>
__global__ void __launch_bounds__(128) fuse_bwd_scatter(const FuseArgs a, const int16_t *__restrict__ crossing,
                                                        const float *__restrict__ grad_fused, float2 *__restrict__ acc) {
    const int i = blockIdx.x * 16 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    if (i >= a.Wt || j >= a.Ht) return;
    const size_t o = (size_t)j * a.Wt + i;
    const int s = crossing[o];
    const float G = grad_fused[o];
    if (s < 0 || s + 1 >= a.D || G == 0.0f) return;
    const float fi = (float)i, fj = (float)j;
    Ray ray[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < a.K) {
            const float *M = a.xf[k].M;
            ray[k].ax = __fmaf_rn(M[0], fi, __fmaf_rn(M[1], fj, M[2]));
            ray[k].ay = __fmaf_rn(M[3], fi, __fmaf_rn(M[4], fj, M[5]));
            ray[k].az = __fmaf_rn(M[6], fi, __fmaf_rn(M[7], fj, M[8]));
        }
    }
    const float z0 = __fmaf_rn((float)s, a.dz, a.zn), z1 = __fmaf_rn((float)(s + 1), a.dz, a.zn);
    float S0, S1, W0, W1;
    evaluate_sample<KMAX, MT>(a, ray, z0, S0, W0);
    evaluate_sample<KMAX, MT>(a, ray, z1, S1, W1);
    const float den = (S0 - S1) * (S0 - S1);
    const float gS[2] = {G * (z1 - z0) * (-S1) / den, G * (z1 - z0) * S0 / den};
    const MT *map = reinterpret_cast<const MT *>(a.dw);
    const size_t plane = (size_t)a.W * a.H;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float zs = t ? z1 : z0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < a.K) {
                const float hz = __fmaf_rn(zs, ray[k].az, a.xf[k].b[2]);
                if (hz > 1e-6f) {
                    const float hx = __fmaf_rn(zs, ray[k].ax, a.xf[k].b[0]);
                    const float hy = __fmaf_rn(zs, ray[k].ay, a.xf[k].b[1]);
                    int u, v;
                    nearest_pixel(hx, hy, hz, u, v);
                    if ((unsigned)u < (unsigned)a.W && (unsigned)v < (unsigned)a.H) {
                        const size_t q = (size_t)k * plane + (size_t)v * a.W + u;
                        const float2 p = load_map(&map[q]);
                        const float sdf = (p.x - hz) * a.inv_mu;
                        if (sdf >= -1.0f && p.y > 0.0f) {
                            const float c = fminf(sdf, 1.0f);
                            const float inband = (sdf > -1.0f && sdf < 1.0f) ? a.inv_mu : 0.0f;
                            atomicAdd(&acc[q], make_float2(gS[t] * c, gS[t] * p.y * inband));
                        }
                    }
                }
            }
        }
    }
}

// Entries e in [-R, R] of a clamp-to-edge window centred at c that land on x
// (one axis, image extent n).
__device__ __forceinline__ int window_multiplicity(int c, int x, int n, int R) {
    if (c < 0 || c >= n) return 0;
    if (n == 1) return 2 * R + 1;
    if (x == 0) return max(0, R - c + 1);
    if (x == n - 1) return max(0, c - (n - 1) + R + 1);
    return abs(c - x) <= R ? 1 : 0;
}

constexpr int GB_TX = 32;
constexpr int GB_TY = 8;

template <int R, typename DT>
__global__ void __launch_bounds__(GB_TX *GB_TY) fuse_bwd_gather(const DT *__restrict__ depth,
                                                                const float2 *__restrict__ acc,
                                                                float *__restrict__ grad, int W, int H, float mu,
                                                                float wconst, float inv_w2) {
    constexpr int DW = GB_TX + 4 * R, DH = GB_TY + 4 * R;   // depths: outputs + 2R halo
    constexpr int PW = GB_TX + 2 * R, PH = GB_TY + 2 * R;   // P(c): outputs + R halo
    __shared__ float dt[DH][DW];
    __shared__ float pt[PH][PW];
    const int k = blockIdx.z;
    const DT *dep = depth + (size_t)k * W * H;
    const float2 *ak = acc + (size_t)k * W * H;
    const int bx = blockIdx.x * GB_TX, by = blockIdx.y * GB_TY;
    const int tid = threadIdx.y * GB_TX + threadIdx.x;
    for (int e = tid; e < DW * DH; e += GB_TX * GB_TY) {
        const int sy = e / DW, sx = e - sy * DW;
        const int gx = min(max(bx - 2 * R + sx, 0), W - 1), gy = min(max(by - 2 * R + sy, 0), H - 1);
        const float d = load_depth(&dep[(size_t)gy * W + gx]);
        dt[sy][sx] = valid_depth(d) ? d : __int_as_float(0x7fc00000);
    }
    __syncthreads();
    // P(c) = A(c) domega/dnu(c) on the outputs and an R halo
    for (int e = tid; e < PW * PH; e += GB_TX * GB_TY) {
        const int py = e / PW, px = e - py * PW;
        const int cx = bx - R + px, cy = by - R + py;
        float P = 0.0f;
        if (cx >= 0 && cx < W && cy >= 0 && cy < H) {
            const float A = ak[(size_t)cy * W + cx].x;
            const float dc = dt[py + R][px + R];
            if (A != 0.0f && dc == dc) {
                float nu = 0.0f;
                for (int dy = 0; dy <= 2 * R; ++dy)
                    for (int dx = 0; dx <= 2 * R; ++dx) {
                        const float t = fminf(fabsf(dc - dt[py + dy][px + dx]), mu);
                        nu = fmaf(t, t, nu);
                    }
                const float unclamped = nu > 0.0f ? wconst * rsqrtf(nu * inv_w2) : 2.0f;
                if (unclamped < 1.0f) P = A * (-0.5f * unclamped / nu);
            }
        }
        pt[py][px] = P;
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= W || y >= H) return;
    const float dx0 = dt[threadIdx.y + 2 * R][threadIdx.x + 2 * R];
    float g = ak[(size_t)y * W + x].y;  // B(x)
    if (dx0 == dx0) {
        const float Px = pt[threadIdx.y + R][threadIdx.x + R];
        if (Px != 0.0f) {
            float sum = 0.0f;
            for (int ey = -R; ey <= R; ++ey)
                for (int ex = -R; ex <= R; ++ex) {
                    const float dn = dt[threadIdx.y + 2 * R + ey][threadIdx.x + 2 * R + ex];
                    const float diff = dx0 - dn;
                    if (fabsf(diff) < mu) sum += 2.0f * diff;  // false for a NaN (invalid) neighbour
                }
            g += Px * sum;
        }
        for (int cyo = -R; cyo <= R; ++cyo) {
            const int my = window_multiplicity(y + cyo, y, H, R);
            if (my == 0) continue;
            for (int cxo = -R; cxo <= R; ++cxo) {
                const int mx = window_multiplicity(x + cxo, x, W, R);
                if (mx == 0) continue;
                const float Pc = pt[threadIdx.y + R + cyo][threadIdx.x + R + cxo];
                if (Pc == 0.0f) continue;
                const float diff = dt[threadIdx.y + 2 * R + cyo][threadIdx.x + 2 * R + cxo] - dx0;
                if (fabsf(diff) < mu) g += (float)(mx * my) * Pc * (-2.0f) * diff;
            }
        }
    }
    grad[(size_t)k * W * H + (size_t)y * W + x] = g;
}

template <int R, typename DT>
cudaError_t launch_bwd_gather_r(const void *depth, const float2 *acc, float *grad, int K, int W, int H, float mu,
                                float wconst, float inv_w2, cudaStream_t st) {
    dim3 grid((W + GB_TX - 1) / GB_TX, (H + GB_TY - 1) / GB_TY, K);
    fuse_bwd_gather<R, DT><<<grid, dim3(GB_TX, GB_TY), 0, st>>>(reinterpret_cast<const DT *>(depth), acc, grad, W, H,
                                                                mu, wconst, inv_w2);
    return cudaGetLastError();
}

template <typename DT>
cudaError_t launch_bwd_gather(const void *depth, const float2 *acc, float *grad, int K, int W, int H, float mu,
                              float wconst, int window, cudaStream_t st) {
    const float inv_w2 = (float)(1.0 / ((double)window * (double)window));
    switch (window / 2) {
        case 0: return launch_bwd_gather_r<0, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 1: return launch_bwd_gather_r<1, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 2: return launch_bwd_gather_r<2, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 3: return launch_bwd_gather_r<3, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 4: return launch_bwd_gather_r<4, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 5: return launch_bwd_gather_r<5, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 6: return launch_bwd_gather_r<6, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 7: return launch_bwd_gather_r<7, DT>(depth, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int R, typename DT, typename MT>
cudaError_t launch_wm(const void *depth, char *map, const MapLayout &L, float mu, float wconst, float inv_w2,
                      cudaStream_t st) {
    dim3 grid((L.W + WM_TX - 1) / WM_TX, (L.H + WM_TY - 1) / WM_TY, L.K);
    weight_map_kernel<R, DT, MT><<<grid, dim3(WM_TX, WM_TY / WM_P), 0, st>>>(reinterpret_cast<const DT *>(depth), map,
                                                                          L, mu, wconst, inv_w2);
    return cudaGetLastError();
}

template <typename DT, typename MT>
cudaError_t launch_wm_window(const void *depth, char *map, const MapLayout &L, float mu, float wconst, int window,
                             cudaStream_t st) {
    const float inv_w2 = (float)(1.0 / ((double)window * (double)window));
    switch (window / 2) {
        case 0: return launch_wm<0, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 1: return launch_wm<1, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 2: return launch_wm<2, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 3: return launch_wm<3, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 4: return launch_wm<4, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 5: return launch_wm<5, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 6: return launch_wm<6, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        case 7: return launch_wm<7, DT, MT>(depth, map, L, mu, wconst, inv_w2, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_weight_map(const void *depth, int depth_dtype, void *map, int map_dtype, int K, int W, int H,
                              float mu, float wconst, int window, cudaStream_t st) {
    if (K == 0) return cudaSuccess;
    const MapLayout L = map_layout(K, W, H);
    char *m = reinterpret_cast<char *>(map);
    cudaError_t e;
    if (depth_dtype == GVS_F16) {
        e = map_dtype == GVS_F16 ? launch_wm_window<__half, __half2>(depth, m, L, mu, wconst, window, st)
                                 : launch_wm_window<__half, float2>(depth, m, L, mu, wconst, window, st);
    } else {
        e = map_dtype == GVS_F16 ? launch_wm_window<float, __half2>(depth, m, L, mu, wconst, window, st)
                                 : launch_wm_window<float, float2>(depth, m, L, mu, wconst, window, st);
    }
    if (e != cudaSuccess) return e;
    depth_bounds_kernel<<<dim3(L.tw[2], L.th[2], K), dim3(16, 16), 0, st>>>(m, L);
    const int64_t n = (int64_t)K * ((int64_t)L.tw[1] * L.th[1] + (int64_t)L.tw[2] * L.th[2]);
    bounds_overlap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, L);
    return cudaGetLastError();
}

cudaError_t launch_fuse_backward(const FuseArgs &a, const void *depth, int depth_dtype, const int16_t *crossing,
                                 const float *grad_fused, float *grad_depths, float2 *acc, float mu, float wconst,
                                 int window, cudaStream_t st) {
    if (a.K == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)a.K * a.W * a.H * sizeof(float2), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.Wt + 15) / 16, (a.Ht + 7) / 8), block(16, 8);
    if (a.map_dtype == GVS_F16) {
        if (a.K <= 4) fuse_bwd_scatter<4, __half2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else if (a.K <= 8) fuse_bwd_scatter<8, __half2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else if (a.K <= 16) fuse_bwd_scatter<16, __half2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else fuse_bwd_scatter<32, __half2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
    } else {
        if (a.K <= 4) fuse_bwd_scatter<4, float2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else if (a.K <= 8) fuse_bwd_scatter<8, float2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else if (a.K <= 16) fuse_bwd_scatter<16, float2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
        else fuse_bwd_scatter<32, float2><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return depth_dtype == GVS_F16
               ? launch_bwd_gather<__half>(depth, acc, grad_depths, a.K, a.W, a.H, mu, wconst, window, st)
               : launch_bwd_gather<float>(depth, acc, grad_depths, a.K, a.W, a.H, mu, wconst, window, st);
}

cudaError_t launch_fuse(const FuseArgs &a, cudaStream_t st) {
    const int64_t nb = (int64_t)((a.Wt + BX - 1) / BX) * ((a.Ht + BY - 1) / BY);
    const unsigned grid = (unsigned)((nb + FZ_WARPS - 1) / FZ_WARPS);
    const dim3 block(32 * FZ_WARPS);
    if (a.map_dtype == GVS_F16) {
        if (a.K <= 4) fuse_kernel<4, __half2><<<grid, block, 0, st>>>(a);
        else if (a.K <= 8) fuse_kernel<8, __half2><<<grid, block, 0, st>>>(a);
        else if (a.K <= 16) fuse_kernel<16, __half2><<<grid, block, 0, st>>>(a);
        else fuse_kernel<32, __half2><<<grid, block, 0, st>>>(a);
    } else {
        if (a.K <= 4) fuse_kernel<4, float2><<<grid, block, 0, st>>>(a);
        else if (a.K <= 8) fuse_kernel<8, float2><<<grid, block, 0, st>>>(a);
        else if (a.K <= 16) fuse_kernel<16, float2><<<grid, block, 0, st>>>(a);
        else fuse_kernel<32, float2><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace gvs
