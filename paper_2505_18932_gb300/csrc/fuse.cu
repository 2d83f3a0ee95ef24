// Image-based TSDF fusion in the target view (Supplement A.1, Eq. 3).
//
// weight_map  : the confidence weight of Supplement A.1 depends only on the
//               sampled input pixel (nearest-pixel sampling), so it is
//               computed once per input pixel and packed with the depth as
//               float2 (d, omega); an invalid pixel is stored as (0, 0), whose
//               signed distance is below -1 so it never contributes.  7x7
//               stencil over a shared-memory tile with halo.  The same kernel
//               writes the bound of every 16x16 tile: smallest and largest
//               valid depth and the mask of occupied depth bins.
// depth_bounds, bounds_overlap: build the per-view bound pyramid (16, 32, 64
//               and 128 pixel tiles, each also as overlapping 2x2-tile
//               blocks, and the whole view) from the 16x16 tiles.
// fuse        : one warp per 8x4 bundle of target pixels, one thread per ray,
//               marching the D samples in registers (one 8-byte gather per
//               sample and view) to the first +/- crossing.  Before evaluating
//               samples the warp tries to prove that a run of them holds no
//               crossing end for any ray of the bundle (see slab_view_free);
//               such runs are skipped.  A skipped sample provably has S > 0 or
//               W = 0, so the first crossing, its index and its interpolated
//               depth are exactly those of the full uniform march.
#include "fuse_march.cuh"

namespace gvs {
namespace {

constexpr int WM_TX = 32;   // block of 32 x 64 output pixels: 32 x 8 threads,
constexpr int WM_P = 8;     // each thread a column of WM_P pixels (8: 3 % faster than 4 at 1080p)
constexpr int WM_TY = 8 * WM_P;

// R = window / 2.  The shared tile holds the block's depths, as the map will
// store them, plus an R-pixel halo replicated at the image borders (invalid
// depths as NaN).  A thread reads each of the (WM_P + 2R) x (2R + 1) shared
// values its column needs once and reuses it for every output whose window
// contains it.  DT: float or __half input; MT: float2 or __half2 map.
// EXACT: omega = min(wconst / sqrt(nu / w^2), 1) with correctly rounded
// operations (bit-reproducible on the host, as the sphere-tracing path needs);
// otherwise with the approximate reciprocal square root.
// 8 resident blocks per SM (32 registers): the stencil needs the warps more
// than the registers (at 51 registers 10 % slower).
template <int R, typename DT, typename MT, bool EXACT = false>
__global__ void __launch_bounds__(256, 8) weight_map_kernel(const DT *__restrict__ depth, char *__restrict__ map,
                                                         MapLayout L, float mu, float wconst, float inv_w2) {
    constexpr int SW = WM_TX + 2 * R;
    constexpr int SH = WM_TY + 2 * R;
    __shared__ float2 tile[SH][SW];  // each depth twice: a ready pair for the packed taps
    __shared__ float2 red[WM_TY / WM_P][WM_TX / 16];
    __shared__ uint2 mred[WM_TY / WM_P][WM_TX / 16];
    const int W = L.W, H = L.H;
    const int k = blockIdx.z;
    const DT *dep = depth + (size_t)k * W * H;
    const int x0 = blockIdx.x * WM_TX - R;
    const int y0 = blockIdx.y * WM_TY - R;
    const int tid = threadIdx.y * WM_TX + threadIdx.x;
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        // whole-view bounds, reduced into by depth_bounds with integer atomics on the float bits
        reinterpret_cast<uint4 *>(map + L.off_g)[k] = make_uint4(0x7f800000u, 0xff800000u, ~0u, ~0u);
    }
    const int tx = threadIdx.x, ty = threadIdx.y;
    {
        // rows of the tile by thread row, columns by lane (a lane's two clamped columns
        // computed once): the loads of all its rows are independent and in flight together
        static_assert(SW - WM_TX <= WM_TX, "the halo columns fit one more pass of the lanes");
        constexpr int TR = WM_TY / WM_P;  // thread rows
        const int gxa = min(max(x0 + tx, 0), W - 1);
        const int gxb = min(max(x0 + WM_TX + tx, 0), W - 1);
        const bool has_b = tx < SW - WM_TX;
#pragma unroll
        for (int sy = ty; sy < SH; sy += TR) {
            const DT *row = dep + (size_t)min(max(y0 + sy, 0), H - 1) * W;
            const float da = as_stored(load_depth(&row[gxa]), (MT *)nullptr);
            const float va = valid_depth(da) ? da : __int_as_float(0x7fc00000);  // NaN marks invalid
            tile[sy][tx] = make_float2(va, va);
            if (has_b) {
                const float db = as_stored(load_depth(&row[gxb]), (MT *)nullptr);
                const float vb = valid_depth(db) ? db : __int_as_float(0x7fc00000);
                tile[sy][WM_TX + tx] = make_float2(vb, vb);
            }
        }
    }
    __syncthreads();
    const int x = blockIdx.x * WM_TX + tx;
    const int yb = blockIdx.y * WM_TY + ty * WM_P;
    // Two vertically adjacent outputs take a neighbour they share in one packed
    // add and one packed FMA: |dc - n| = |n + (-dc)| exactly, and each output
    // still sums its taps in the same order with the same roundings.
    static_assert(WM_P % 2 == 0, "outputs are paired");
    float dc[WM_P];
    float2 ndc[WM_P / 2], nu[WM_P / 2];
#pragma unroll
    for (int p = 0; p < WM_P; ++p) dc[p] = tile[ty * WM_P + p + R][tx + R].x;
#pragma unroll
    for (int q = 0; q < WM_P / 2; ++q) {
        ndc[q] = make_float2(-dc[2 * q], -dc[2 * q + 1]);
        nu[q] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int r = 0; r < WM_P + 2 * R; ++r) {
        float2 row[2 * R + 1];
#pragma unroll
        for (int dx = 0; dx <= 2 * R; ++dx) row[dx] = tile[ty * WM_P + r][tx + dx];
#pragma unroll
        for (int q = 0; q < WM_P / 2; ++q) {
            const bool in0 = r - 2 * q >= 0 && r - 2 * q <= 2 * R;
            const bool in1 = r - 2 * q - 1 >= 0 && r - 2 * q - 1 <= 2 * R;
#pragma unroll
            for (int dx = 0; dx <= 2 * R; ++dx) {
                // fminf returns mu for a NaN (invalid) neighbour: it counts mu^2
                if (in0 && in1) {
                    const float2 e = __fadd2_rn(row[dx], ndc[q]);
                    const float2 t = make_float2(fminf(fabsf(e.x), mu), fminf(fabsf(e.y), mu));
                    nu[q] = __ffma2_rn(t, t, nu[q]);
                } else if (in0) {
                    const float t = fminf(fabsf(row[dx].x + ndc[q].x), mu);
                    nu[q].x = fmaf(t, t, nu[q].x);
                } else if (in1) {
                    const float t = fminf(fabsf(row[dx].y + ndc[q].y), mu);
                    nu[q].y = fmaf(t, t, nu[q].y);
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
                const float n = (p & 1) ? nu[p >> 1].y : nu[p >> 1].x;
                if (EXACT)
                    w = n > 0.0f ? fminf(__fdiv_rn(wconst, __fsqrt_rn(__fmul_rn(n, inv_w2))), 1.0f) : 1.0f;
                else
                    w = n > 0.0f ? fminf(wconst * rsqrtf(n * inv_w2), 1.0f) : 1.0f;
                d = dc[p];
                lo = fminf(lo, d);
                hi = fmaxf(hi, d);
            }
            store_map(&dw[(size_t)y * W + x], d, w);
        }
    }
    // 16x16 tile bounds: over the 16 lanes of a tile's columns, then its two thread rows
    static_assert(WM_P == 8 && WM_TX % 16 == 0 && WM_TY % 16 == 0, "a 16x16 tile is 16 lanes x 2 thread rows");
#pragma unroll
    for (int m = 1; m < 16; m <<= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, m));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, m));
    }
    if ((tx & 15) == 0) red[ty][tx >> 4] = make_float2(lo, hi);
    __syncthreads();
    const float tlo = fminf(red[ty & ~1][tx >> 4].x, red[ty | 1][tx >> 4].x);
    const float thi = fmaxf(red[ty & ~1][tx >> 4].y, red[ty | 1][tx >> 4].y);
    // the tile's mask: the bin of every valid depth in it, relative to the bin of the smallest
    unsigned long long mask = 0;
    const int base = depth_bin(tlo);
#pragma unroll
    for (int p = 0; p < WM_P; ++p)
        if (x < W && yb + p < H && dc[p] == dc[p]) mask |= 1ull << min(depth_bin(dc[p]) - base, kDepthBins - 1);
    unsigned mlo = (unsigned)mask, mhi = (unsigned)(mask >> 32);
#pragma unroll
    for (int m = 1; m < 16; m <<= 1) {
        mlo |= __shfl_xor_sync(0xffffffffu, mlo, m);
        mhi |= __shfl_xor_sync(0xffffffffu, mhi, m);
    }
    if ((tx & 15) == 0) mred[ty][tx >> 4] = make_uint2(mlo, mhi);
    __syncthreads();
    if ((tx & 15) == 0 && (ty & 1) == 0) {
        const uint2 o = mred[ty | 1][tx >> 4];
        const int gx = blockIdx.x * (WM_TX / 16) + (tx >> 4), gy = blockIdx.y * (WM_TY / 16) + (ty >> 1);
        if (gx < L.tw[0] && gy < L.th[0])
            reinterpret_cast<uint4 *>(map + L.off_T[0])[((size_t)k * L.th[0] + gy) * L.tw[0] + gx] =
                make_uint4(__float_as_uint(tlo), __float_as_uint(thi), mlo | o.x, mhi | o.y);
    }
}

__device__ __forceinline__ DepthBound empty_bound() {
    DepthBound b;
    b.lo = kInf;
    b.hi = -kInf;
    b.mlo = b.mhi = 0u;
    return b;
}

__device__ __forceinline__ DepthBound load_bound(const DepthBound *p) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p);
    DepthBound b;
    b.lo = __uint_as_float(v.x);
    b.hi = __uint_as_float(v.y);
    b.mlo = v.z;
    b.mhi = v.w;
    return b;
}

__device__ __forceinline__ void store_bound(DepthBound *p, const DepthBound &b) {
    *reinterpret_cast<uint4 *>(p) = make_uint4(__float_as_uint(b.lo), __float_as_uint(b.hi), b.mlo, b.mhi);
}

// A child's mask in the bins of a parent whose smallest depth lies sh >= 0 bins
// lower: bins moved past 63 land on 63.
__device__ __forceinline__ unsigned long long shift_bins(unsigned long long m, int sh) {
    if (m == 0ull) return 0ull;
    if (sh >= 64) return 1ull << 63;
    if (sh == 0) return m;
    return (m << sh) | ((m >> (64 - sh)) ? (1ull << 63) : 0ull);
}

__device__ __forceinline__ void rebin_into(DepthBound &p, const DepthBound &c) {
    if (!(c.lo <= c.hi)) return;  // no valid depth in c
    const unsigned long long m =
        shift_bins(((unsigned long long)c.mhi << 32) | c.mlo, depth_bin(c.lo) - depth_bin(p.lo));
    p.mlo |= (unsigned)m;
    p.mhi |= (unsigned)(m >> 32);
}

__device__ __forceinline__ DepthBound merge4(const DepthBound &a, const DepthBound &b, const DepthBound &c,
                                             const DepthBound &d) {
    DepthBound p;
    p.lo = fminf(fminf(a.lo, b.lo), fminf(c.lo, d.lo));
    p.hi = fmaxf(fmaxf(a.hi, b.hi), fmaxf(c.hi, d.hi));
    p.mlo = p.mhi = 0u;
    if (p.lo <= p.hi) {
        rebin_into(p, a);
        rebin_into(p, b);
        rebin_into(p, c);
        rebin_into(p, d);
    }
    return p;
}

// One block per (128x128 pixel tile, view), one thread per 16x16 tile of it:
// writes O_4 (needs one tile of halo right and below), T_5, T_6, T_7 and the
// view bounds.
__global__ void __launch_bounds__(64) depth_bounds_kernel(char *__restrict__ map, MapLayout L) {
    __shared__ DepthBound s4[9][9];
    __shared__ DepthBound s5[4][4];
    __shared__ DepthBound s6[2][2];
    const int k = blockIdx.z;
    const DepthBound *T4 = reinterpret_cast<const DepthBound *>(map + L.off_T[0]) + (size_t)k * L.tw[0] * L.th[0];
    const int x = threadIdx.x, y = threadIdx.y;
    const int tid = y * 8 + x;
    for (int e = tid; e < 9 * 9; e += 64) {
        const int ly = e / 9, lx = e - ly * 9;
        const int tx = blockIdx.x * 8 + lx, ty = blockIdx.y * 8 + ly;
        s4[ly][lx] = (tx < L.tw[0] && ty < L.th[0]) ? load_bound(&T4[(size_t)ty * L.tw[0] + tx]) : empty_bound();
    }
    __syncthreads();
    {
        const int tx = blockIdx.x * 8 + x, ty = blockIdx.y * 8 + y;
        if (tx < L.tw[0] && ty < L.th[0])
            store_bound(reinterpret_cast<DepthBound *>(map + L.off_O[0]) + ((size_t)k * L.th[0] + ty) * L.tw[0] + tx,
                        merge4(s4[y][x], s4[y][x + 1], s4[y + 1][x], s4[y + 1][x + 1]));
    }
    if (x < 4 && y < 4) {
        const DepthBound b = merge4(s4[2 * y][2 * x], s4[2 * y][2 * x + 1], s4[2 * y + 1][2 * x],
                                    s4[2 * y + 1][2 * x + 1]);
        s5[y][x] = b;
        const int tx = blockIdx.x * 4 + x, ty = blockIdx.y * 4 + y;
        if (tx < L.tw[1] && ty < L.th[1])
            store_bound(reinterpret_cast<DepthBound *>(map + L.off_T[1]) + ((size_t)k * L.th[1] + ty) * L.tw[1] + tx, b);
    }
    __syncthreads();
    if (x < 2 && y < 2) {
        const DepthBound b = merge4(s5[2 * y][2 * x], s5[2 * y][2 * x + 1], s5[2 * y + 1][2 * x],
                                    s5[2 * y + 1][2 * x + 1]);
        s6[y][x] = b;
        const int tx = blockIdx.x * 2 + x, ty = blockIdx.y * 2 + y;
        if (tx < L.tw[2] && ty < L.th[2])
            store_bound(reinterpret_cast<DepthBound *>(map + L.off_T[2]) + ((size_t)k * L.th[2] + ty) * L.tw[2] + tx, b);
    }
    __syncthreads();
    if (tid == 0) {
        const DepthBound b = merge4(s6[0][0], s6[0][1], s6[1][0], s6[1][1]);
        store_bound(reinterpret_cast<DepthBound *>(map + L.off_T[3]) +
                        ((size_t)k * L.th[3] + blockIdx.y) * L.tw[3] + blockIdx.x, b);
        unsigned *g = reinterpret_cast<unsigned *>(reinterpret_cast<DepthBound *>(map + L.off_g) + k);
        if (b.lo <= b.hi) {  // the tile holds a valid depth; positive floats order like their bits
            atomicMin(&g[0], __float_as_uint(b.lo));
            atomicMax(&g[1], __float_as_uint(b.hi));
        }
    }
}

// O_l from T_l for levels 5, 6 and 7: one thread per (view, tile).
__global__ void __launch_bounds__(256) bounds_overlap_kernel(char *__restrict__ map, MapLayout L) {
    int64_t n[kBoundLevels], total = 0;
    for (int l = 1; l < kBoundLevels; ++l) {
        n[l] = (int64_t)L.tw[l] * L.th[l];
        total += n[l];
    }
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)L.K * total) return;
    const int k = (int)(q / total);
    q -= (int64_t)k * total;
    int l = 1;
    while (q >= n[l]) q -= n[l++];
    const int tw = L.tw[l], th = L.th[l];
    const int tx = (int)(q % tw), ty = (int)(q / tw);
    const DepthBound *T = reinterpret_cast<const DepthBound *>(map + L.off_T[l]) + (size_t)k * tw * th;
    const DepthBound e = empty_bound();
    const DepthBound a = load_bound(&T[(size_t)ty * tw + tx]);
    const DepthBound b = tx + 1 < tw ? load_bound(&T[(size_t)ty * tw + tx + 1]) : e;
    const DepthBound c = ty + 1 < th ? load_bound(&T[(size_t)(ty + 1) * tw + tx]) : e;
    const DepthBound d = (tx + 1 < tw && ty + 1 < th) ? load_bound(&T[(size_t)(ty + 1) * tw + tx + 1]) : e;
    store_bound(reinterpret_cast<DepthBound *>(map + L.off_O[l]) + ((size_t)k * th + ty) * tw + tx, merge4(a, b, c, d));
}

template <int KMAX, typename MT, typename T, bool TMP>
__global__ void __launch_bounds__(32 * FZ_WARPS, GVS_FUSE_MIN_BLOCKS) fuse_kernel(const __grid_constant__ FuseArgs a) {
    const int nbundles = ((a.Wt + T::bx - 1) / T::bx) * ((a.Ht + T::by - 1) / T::by);
    const int bundle = blockIdx.x * FZ_WARPS + (threadIdx.x >> 5);
    if (bundle >= nbundles) return;  // the whole warp leaves together
    march_bundle<KMAX, MT, T, TMP>(a, bundle, threadIdx.x & 31);
}

template <int KMAX, typename MT, typename T, bool TMP>
void launch_fuse_t(const FuseArgs &a, cudaStream_t st) {
    const int64_t nb = (int64_t)((a.Wt + T::bx - 1) / T::bx) * ((a.Ht + T::by - 1) / T::by);
    fuse_kernel<KMAX, MT, T, TMP><<<(unsigned)((nb + FZ_WARPS - 1) / FZ_WARPS), 32 * FZ_WARPS, 0, st>>>(a);
}

template <int KMAX, typename MT, typename T>
struct FuseLaunch {
    static void run(const FuseArgs &a, cudaStream_t st) { launch_fuse_t<KMAX, MT, T, false>(a, st); }
};

// With the temporal input (Supplement A.2): the default tile only.
template <int KMAX, typename MT, typename T>
struct FuseLaunchTemporal {
    static void run(const FuseArgs &a, cudaStream_t st) { launch_fuse_t<KMAX, MT, T, true>(a, st); }
};
template <int R, typename DT, typename MT>
cudaError_t launch_wm(const void *depth, char *map, const MapLayout &L, float mu, float wconst, float inv_w2,
                      bool exact, cudaStream_t st) {
    dim3 grid((L.W + WM_TX - 1) / WM_TX, (L.H + WM_TY - 1) / WM_TY, L.K);
    if (exact)
        weight_map_kernel<R, DT, MT, true><<<grid, dim3(WM_TX, WM_TY / WM_P), 0, st>>>(
            reinterpret_cast<const DT *>(depth), map, L, mu, wconst, inv_w2);
    else
        weight_map_kernel<R, DT, MT><<<grid, dim3(WM_TX, WM_TY / WM_P), 0, st>>>(reinterpret_cast<const DT *>(depth),
                                                                              map, L, mu, wconst, inv_w2);
    return cudaGetLastError();
}

template <typename DT, typename MT>
cudaError_t launch_wm_window(const void *depth, char *map, const MapLayout &L, float mu, float wconst, int window,
                             bool exact, cudaStream_t st) {
    const float inv_w2 = (float)(1.0 / ((double)window * (double)window));
    switch (window / 2) {
        case 0: return launch_wm<0, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 1: return launch_wm<1, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 2: return launch_wm<2, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 3: return launch_wm<3, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 4: return launch_wm<4, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 5: return launch_wm<5, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 6: return launch_wm<6, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        case 7: return launch_wm<7, DT, MT>(depth, map, L, mu, wconst, inv_w2, exact, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_weight_map(const void *depth, int depth_dtype, void *map, int map_dtype, int K, int W, int H,
                              float mu, float wconst, int window, cudaStream_t st, bool exact) {
    if (K == 0) return cudaSuccess;
    const MapLayout L = map_layout(K, W, H);
    char *m = reinterpret_cast<char *>(map);
    cudaError_t e;
    if (depth_dtype == GVS_F16) {
        e = map_dtype == GVS_F16 ? launch_wm_window<__half, __half2>(depth, m, L, mu, wconst, window, false, st)
                                 : launch_wm_window<__half, float2>(depth, m, L, mu, wconst, window, exact, st);
    } else {
        e = map_dtype == GVS_F16 ? launch_wm_window<float, __half2>(depth, m, L, mu, wconst, window, false, st)
                                 : launch_wm_window<float, float2>(depth, m, L, mu, wconst, window, exact, st);
    }
    if (e != cudaSuccess) return e;
    depth_bounds_kernel<<<dim3(L.tw[3], L.th[3], K), dim3(8, 8), 0, st>>>(m, L);
    int64_t n = 0;
    for (int l = 1; l < kBoundLevels; ++l) n += (int64_t)L.tw[l] * L.th[l];
    n *= K;
    bounds_overlap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, L);
    return cudaGetLastError();
}

int bundle_count(int Wt, int Ht, int K, int variant) {
    if (K > 4 && variant == 6) return Wt * Ht;  // one warp per ray (the 8, 16 and 32-view kernels)
    int bx = 8, by = 4;
    if (K > 4 && K <= 16) {
        if (variant == 2) { bx = 16; by = 2; }
        else if (variant == 3 || variant == 4) { bx = 4; by = 8; }
    }
    return ((Wt + bx - 1) / bx) * ((Ht + by - 1) / by);
}

cudaError_t launch_fuse(const FuseArgs &a, cudaStream_t st) {
    if (a.tmp_depth || a.wview)
        by_kmax_tile0<FuseLaunchTemporal>(a.K, a.map_dtype, a, st);
    else
        by_kmax<FuseLaunch>(a.K, a.map_dtype, a.variant, a, st);
    return cudaGetLastError();
}

GVS_BOUNDS_TAKE_FN(bounds_take_fuse)

}  // namespace gvs
