// Pixel-sized Gaussian forward render (Sec. 3.1, Supplement A.3), each input
// view separately, with the rasterisation rules of 3D Gaussian splatting
// (Kerbl et al. 2023) restated for isotropic, fully opaque Gaussians:
//   prep   : one thread per source pixel.  Splat contract for the mean
//            (x, y) and depth z; EWA covariance
//              Sigma = (scale rho)^2 [[1 + a^2, q a b], [q a b, q^2 (1 + b^2)]] + 0.3 I
//            (rho = f (d / z), a = (x - cx) / fx, b = (y - cy) / fy, q = fy / fx);
//            radius r = min(ceil(3 sqrt(lambda_max)), max_radius), narrowed
//            to where alpha can reach 1/255 (see GaussRec); the record
//            (x, y, z, half-widths | conic, colour); one counter increment per
//            16 x 16 target tile its box meets (warp-aggregated atomics).
//   scan   : exclusive scan of the tile counters -> list offsets.
//   fill   : each Gaussian writes its key (bits(z) << 32 | source index) into
//            the list of every tile it meets.
//   render : one block per tile.  The list is sorted ascending (bitonic, in
//            shared memory up to GS_SORT_CAP keys, else in place in global
//            memory), then every thread composites its pixel front to back:
//            alpha = min(0.99, exp(power)), skipped below 1/255, stop before
//            a Gaussian that would take T below 1e-4.
// The radius, the box and the key are integer decisions taken with explicitly
// rounded FP32 operations (no contraction), exactly as the header states them.
#include <cuda_fp16.h>
#include <math.h>

#include "bounds_check.cuh"
#include "gauss_internal.cuh"

namespace gvs {
namespace {

constexpr int GS_THREADS = GS_TILE * GS_TILE;

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.0f; }
__device__ __forceinline__ float load_depth(const float *p) { return __ldg(p); }
__device__ __forceinline__ float load_depth(const __half *p) { return __half2float(__ldg(p)); }

// a.w holds the half-widths (hx, hy) of the Gaussian's box as a half2 (bits 0:
// no Gaussian): the contract radius r, tightened to the extent of the ellipse
// where alpha can reach 1/255, sqrt(2 ln 255 Sigma_xx) (and yy), widened by
// 0.1 % + 1e-3 px and rounded up.  A pixel between that box and the contract's
// [x - r, x + r] box has alpha below 1/255 by more than 1 % and is skipped by
// both, so the narrower box changes no result; it only shortens the lists.
struct GaussRec {
    float4 a;  // x, y, z, half2 (hx, hy)
    float4 b;  // -conic_xx / 2, -conic_xy, -conic_yy / 2, colour bits
};

__device__ __forceinline__ float2 half_widths(float w) {
    const unsigned bits = __float_as_uint(w);
    return __half22float2(*reinterpret_cast<const __half2 *>(&bits));
}

// Warp-aggregated atomicAdd of 1 on ctr[t]: lanes adding to the same counter
// share one atomic; each gets a distinct old value.
__device__ __forceinline__ unsigned agg_increment(unsigned *ctr, int t) {
    const unsigned peers = __match_any_sync(__activemask(), t);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&ctr[t], (unsigned)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__device__ __forceinline__ GaussRec *recs(const GaussArgs &g) {
    return reinterpret_cast<GaussRec *>(g.ws + g.L.off_rec);
}

// Target pixels of a record's box: [ceil(x - hx), floor(x + hx)] clipped (and y alike).
__device__ __forceinline__ bool box_of(const GaussArgs &g, float4 a, int &i0, int &i1, int &j0, int &j1) {
    if (__float_as_uint(a.w) == 0u) return false;
    const float2 h = half_widths(a.w);
    float lx = ceilf(__fsub_rn(a.x, h.x)), hx = floorf(__fadd_rn(a.x, h.x));
    float ly = ceilf(__fsub_rn(a.y, h.y)), hy = floorf(__fadd_rn(a.y, h.y));
    if (lx < 0.0f) lx = 0.0f;
    if (ly < 0.0f) ly = 0.0f;
    if (hx > (float)(g.Wt - 1)) hx = (float)(g.Wt - 1);
    if (hy > (float)(g.Ht - 1)) hy = (float)(g.Ht - 1);
    if (!(lx <= hx) || !(ly <= hy)) return false;
    i0 = (int)lx; i1 = (int)hx; j0 = (int)ly; j1 = (int)hy;
    return true;
}

template <typename DT>
__global__ void __launch_bounds__(256) gauss_prep(const GaussArgs g, int k) {
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    const int src = v * g.W + u;
    const size_t HW = (size_t)g.W * g.H;
    const float d = load_depth(reinterpret_cast<const DT *>(g.depth) + (size_t)k * HW + src);
    GaussRec r;
    r.a = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    r.b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (valid_depth(d)) {
        const float *A = g.xf[k].M, *c = g.xf[k].b;
        const float fu = (float)u, fv = (float)v;
        const float m0 = __fmaf_rn(A[0], fu, __fmaf_rn(A[1], fv, A[2]));
        const float m1 = __fmaf_rn(A[3], fu, __fmaf_rn(A[4], fv, A[5]));
        const float m2 = __fmaf_rn(A[6], fu, __fmaf_rn(A[7], fv, A[8]));
        const float h0 = __fmaf_rn(d, m0, c[0]);
        const float h1 = __fmaf_rn(d, m1, c[1]);
        const float h2 = __fmaf_rn(d, m2, c[2]);
        if (h2 > 1e-6f) {
            const float x = __fdiv_rn(h0, h2), y = __fdiv_rn(h1, h2);
            const float rho = __fmul_rn(g.f_ratio[k], __fdiv_rn(d, h2));
            const float t = __fmul_rn(g.scale_px, rho);
            const float s2 = __fmul_rn(t, t);
            const float ea = __fdiv_rn(__fsub_rn(x, g.in32[2]), g.in32[0]);
            const float eb = __fdiv_rn(__fsub_rn(y, g.in32[3]), g.in32[1]);
            const float q = g.in32[4];
            const float aa = __fmul_rn(ea, ea), bb = __fmul_rn(eb, eb), ab = __fmul_rn(ea, eb);
            const float qq = __fmul_rn(q, q);
            const float sxx = __fadd_rn(__fmul_rn(s2, __fadd_rn(1.0f, aa)), 0.3f);
            const float sxy = __fmul_rn(s2, __fmul_rn(q, ab));
            const float syy = __fadd_rn(__fmul_rn(s2, __fmul_rn(qq, __fadd_rn(1.0f, bb))), 0.3f);
            const float det = __fsub_rn(__fmul_rn(sxx, syy), __fmul_rn(sxy, sxy));
            if (det > 0.0f) {
                const float mid = __fmul_rn(0.5f, __fadd_rn(sxx, syy));
                float disc = __fsub_rn(__fmul_rn(mid, mid), det);
                disc = disc > 0.1f ? disc : 0.1f;
                const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
                float rr = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
                if (!(rr <= (float)g.max_radius)) rr = (float)g.max_radius;
                const float ex = fmaf(sqrtf(11.0825271f * sxx), 1.001f, 1e-3f);  // 2 ln 255 = 11.0825271
                const float ey = fmaf(sqrtf(11.0825271f * syy), 1.001f, 1e-3f);
                const __half2 hw = __halves2half2(__float2half_ru(fminf(ex, rr)), __float2half_ru(fminf(ey, rr)));
                r.a = make_float4(x, y, h2, __uint_as_float(*reinterpret_cast<const unsigned *>(&hw)));
                const float inv = 1.0f / det;
                r.b = make_float4(-0.5f * syy * inv, sxy * inv, -0.5f * sxx * inv,
                                  __uint_as_float(__ldg(&g.rgba[(size_t)k * HW + src])));
            }
        }
    }
    int i0, i1, j0, j1;
    const bool any = box_of(g, r.a, i0, i1, j0, j1);
    if (!any) r.a.w = 0.0f;
    recs(g)[src] = r;
    if (any) {
        unsigned *count = reinterpret_cast<unsigned *>(g.ws + g.L.off_count);
        for (int ty = j0 / GS_TILE; ty <= j1 / GS_TILE; ++ty)
            for (int tx = i0 / GS_TILE; tx <= i1 / GS_TILE; ++tx) agg_increment(count, ty * g.L.tiles_x + tx);
    }
}

// Single block: exclusive scan of the tile counters into 64-bit offsets
// (offset[nt] = total); the counters are reset to serve as fill cursors.
__global__ void __launch_bounds__(1024) gauss_scan(GaussArgs g) {
    const int nt = g.L.tiles_x * g.L.tiles_y;
    unsigned *count = reinterpret_cast<unsigned *>(g.ws + g.L.off_count);
    unsigned long long *off = reinterpret_cast<unsigned long long *>(g.ws + g.L.off_offset);
    __shared__ unsigned long long warp_sum[32];
    const int tid = threadIdx.x;
    const int per = (nt + 1023) / 1024;
    const int b0 = tid * per, b1 = min(b0 + per, nt);
    unsigned long long s = 0;
    for (int t = b0; t < b1; ++t) s += count[t];
    // inclusive scan of s over the block
    unsigned long long x = s;
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, m);
        if (lane >= m) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long z = warp_sum[lane];
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, z, m);
            if (lane >= m) z += y;
        }
        warp_sum[lane] = z;
    }
    __syncthreads();
    unsigned long long run = x - s + (w > 0 ? warp_sum[w - 1] : 0ull);
    for (int t = b0; t < b1; ++t) {
        off[t] = run;
        run += count[t];
        count[t] = 0u;
    }
    if (tid == 1023) off[nt] = run;
}

__global__ void __launch_bounds__(256) gauss_fill(const GaussArgs g) {
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 8 + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    const int src = v * g.W + u;
    const float4 a = recs(g)[src].a;
    int i0, i1, j0, j1;
    if (!box_of(g, a, i0, i1, j0, j1)) return;
    unsigned *cursor = reinterpret_cast<unsigned *>(g.ws + g.L.off_count);
    const unsigned long long *off = reinterpret_cast<const unsigned long long *>(g.ws + g.L.off_offset);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(g.ws + g.L.off_keys);
    const unsigned long long key = ((unsigned long long)__float_as_uint(a.z) << 32) | (unsigned)src;
    for (int ty = j0 / GS_TILE; ty <= j1 / GS_TILE; ++ty)
        for (int tx = i0 / GS_TILE; tx <= i1 / GS_TILE; ++tx) {
            const int t = ty * g.L.tiles_x + tx;
            const unsigned long long pos = off[t] + agg_increment(cursor, t);
            if (GVS_IN_BOUNDS(pos, g.L.n_keys, GVS_SITE_GAUSS_KEY)) keys[pos] = key;
        }
}

// Ascending bitonic sort of key[0, n) by the block; positions n.. act as +inf
// padding up to the next power of two and are never touched (every compare
// puts the smaller key at the lower index).  K: shared or global memory.
__device__ void block_sort(unsigned long long *key, int n) {
    int N = 1, lg = 0;
    while (N < n) { N <<= 1; ++lg; }
    for (int lk = 1; lk <= lg; ++lk) {
        const int hk = 1 << (lk - 1);
        // first step of the merge: compare mirrored positions of each block of 2 hk
        for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
            const int blk = i >> (lk - 1), p = i & (hk - 1);
            const int x = (blk << lk) + p, y = (blk << lk) + (2 * hk - 1 - p);
            if (y < n) {
                const unsigned long long kx = key[x], ky = key[y];
                if (kx > ky) { key[x] = ky; key[y] = kx; }
            }
        }
        __syncthreads();
        for (int lj = lk - 2; lj >= 0; --lj) {
            const int j = 1 << lj;
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                const int x = ((i >> lj) << (lj + 1)) + (i & (j - 1)), y = x + j;
                if (y < n) {
                    const unsigned long long kx = key[x], ky = key[y];
                    if (kx > ky) { key[x] = ky; key[y] = kx; }
                }
            }
            __syncthreads();
        }
    }
}

// Threads of a block: 8 warps, each an 8 x 4 rectangle of the 16 x 16 tile
// (2 across, 4 down).  Per batch of 256 sorted Gaussians every warp first
// compacts, in order, the ones whose box meets its rectangle, then each lane
// walks that shorter list for its pixel.
__global__ void __launch_bounds__(GS_THREADS) gauss_render(const GaussArgs g, int k) {
    __shared__ unsigned long long skeys[GS_SORT_CAP];
    __shared__ float4 sa[GS_THREADS], sb[GS_THREADS], sc[GS_THREADS];
    __shared__ unsigned char wlist[GS_THREADS / 32][GS_THREADS];
    const int t = blockIdx.y * g.L.tiles_x + blockIdx.x;
    const unsigned long long *off = reinterpret_cast<const unsigned long long *>(g.ws + g.L.off_offset);
    unsigned long long *gkeys = reinterpret_cast<unsigned long long *>(g.ws + g.L.off_keys) + off[t];
    const int n = (int)(off[t + 1] - off[t]);
    unsigned long long *keys = gkeys;
    if (n <= GS_SORT_CAP) {
        for (int e = threadIdx.x; e < n; e += GS_THREADS) skeys[e] = gkeys[e];
        keys = skeys;
    }
    __syncthreads();
    block_sort(keys, n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rx = blockIdx.x * GS_TILE + (warp & 1) * 8, ry = blockIdx.y * GS_TILE + (warp >> 1) * 4;
    const int i = rx + (lane & 7);
    const int j = ry + (lane >> 3);
    const bool inside = i < g.Wt && j < g.Ht;
    const float rx0 = (float)rx, rx1 = (float)(rx + 7), ry0 = (float)ry, ry1 = (float)(ry + 3);
    const float fi = (float)i, fj = (float)j;
    bool done = !inside;
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, zs = 0.0f, ws = 0.0f;
    const GaussRec *rec = recs(g);
    for (int b0 = 0; b0 < n; b0 += GS_THREADS) {
        if (__syncthreads_count(!done) == 0) break;  // also orders the reuse of sa / sb
        const int e = b0 + threadIdx.x;
        if (e < n) {
            unsigned src = (unsigned)(keys[e] & 0xffffffffull);
            if (!GVS_IN_BOUNDS(src, (size_t)g.W * g.H, GVS_SITE_GAUSS_REC)) src = 0;
            const GaussRec r = rec[src];
            sa[threadIdx.x] = r.a;
            sb[threadIdx.x] = r.b;
            const unsigned col = __float_as_uint(r.b.w);
            sc[threadIdx.x] = make_float4((float)(col & 0xffu) * (1.0f / 255.0f),
                                          (float)((col >> 8) & 0xffu) * (1.0f / 255.0f),
                                          (float)((col >> 16) & 0xffu) * (1.0f / 255.0f), 0.0f);
        }
        __syncthreads();
        const int m = min(GS_THREADS, n - b0);
        // the Gaussians of this batch whose box meets the warp's rectangle (same rounded
        // bounds as the per-pixel test, so none that covers one of its pixels is dropped)
        int cnt = 0;
        for (int base = 0; base < m; base += 32) {
            const int q = base + lane;
            bool hit = false;
            if (q < m) {
                const float4 a = sa[q];
                const float2 h = half_widths(a.w);
                hit = !(rx1 < __fsub_rn(a.x, h.x) || rx0 > __fadd_rn(a.x, h.x) || ry1 < __fsub_rn(a.y, h.y) ||
                        ry0 > __fadd_rn(a.y, h.y));
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) wlist[warp][cnt + __popc(bal & ((1u << lane) - 1u))] = (unsigned char)q;
            cnt += __popc(bal);
        }
        __syncwarp();
        for (int e = 0; e < cnt; ++e) {
            if (__all_sync(0xffffffffu, done)) break;
            const int q = wlist[warp][e];
            const float4 a = sa[q];
            const float2 h = half_widths(a.w);
            const bool inbox = !(fi < __fsub_rn(a.x, h.x) || fi > __fadd_rn(a.x, h.x) || fj < __fsub_rn(a.y, h.y) ||
                                 fj > __fadd_rn(a.y, h.y));
            const float4 c = sb[q];
            const float dx = a.x - fi, dy = a.y - fj;
            const float power = fmaf(dx, fmaf(c.x, dx, c.y * dy), c.z * dy * dy);
            // exp(-5.6) < 1/255 whatever the rounding of the exponential: skip without it
            const float al = fminf(0.99f, __expf(power));
            const bool use = !done && inbox && !(power > 0.0f || power < -5.6f) && !(al < 1.0f / 255.0f);
            const float Tn = T * (1.0f - al);
            const bool stop = use && Tn < 1e-4f;
            done = done || stop;
            const bool acc = use && !stop;
            const float wgt = acc ? al * T : 0.0f;  // adding 0 leaves every sum as it was
            const float4 cc = sc[q];
            cr = fmaf(cc.x, wgt, cr);
            cg = fmaf(cc.y, wgt, cg);
            cb = fmaf(cc.z, wgt, cb);
            zs = fmaf(a.z, wgt, zs);
            ws += wgt;
            T = acc ? Tn : T;
        }
    }
    if (inside) {
        const size_t o = (size_t)k * g.Wt * g.Ht + (size_t)j * g.Wt + i;
        g.color[o] = make_float4(cr, cg, cb, 1.0f - T);
        g.depth_out[o] = ws > 0.0f ? zs / ws : 0.0f;
    }
}

}  // namespace

cudaError_t launch_gauss_splat(const GaussArgs &a, int K, cudaStream_t st) {
    const GaussLayout &L = a.L;
    const dim3 pg((unsigned)((a.W + 31) / 32), (unsigned)((a.H + 7) / 8)), pb(32, 8);
    const dim3 rg((unsigned)L.tiles_x, (unsigned)L.tiles_y);
    const size_t nt = (size_t)L.tiles_x * L.tiles_y;
    for (int k = 0; k < K; ++k) {
        cudaError_t e = cudaMemsetAsync(a.ws + L.off_count, 0, nt * 4, st);
        if (e != cudaSuccess) return e;
        if (a.depth_dtype == GVS_F16) gauss_prep<__half><<<pg, pb, 0, st>>>(a, k);
        else gauss_prep<float><<<pg, pb, 0, st>>>(a, k);
        gauss_scan<<<1, 1024, 0, st>>>(a);
        gauss_fill<<<pg, pb, 0, st>>>(a);
        gauss_render<<<rg, GS_THREADS, 0, st>>>(a, k);
    }
    return cudaGetLastError();
}

GVS_BOUNDS_TAKE_FN(bounds_take_gauss)

}  // namespace gvs
