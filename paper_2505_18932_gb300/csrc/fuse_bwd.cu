// Adjoint of the image-based TSDF fusion (Supplement A.1, Eq. 3 differentiated).
#include "fuse_march.cuh"

namespace gvs {
namespace {

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
// invalid).  With omega = w_c (nu / w^2)^(-1/2) unsaturated, domega/dnu =
// -0.5 omega / nu = -0.5 omega^3 / (w^2 w_c^2), so a float2 map gives P(c)
// from its stored omega without re-summing the window; for a half2 map (omega
// rounded to half) nu is re-summed from the depths.  Nothing of size D x H x W
// is stored; the bracketing samples are recomputed by the forward's own code,
// so they are bit-identical to it.
// ---------------------------------------------------------------------------

// One target pixel with a crossing: recompute its two bracketing samples and
// add each contributing view's terms at the sampled input pixel.
template <int KMAX, typename MT, bool FULL>
__device__ __forceinline__ void bwd_pixel(const FuseArgs &a, int i, int j, int s, float G, float2 *__restrict__ acc) {
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
    const float z0 = __fmaf_rn((float)s, a.dz, a.zn), z1 = __fmaf_rn((float)(s + 1), a.dz, a.zn);
    float S0, S1, W0, W1;
    evaluate_sample<KMAX, MT, FULL>(a, ray, z0, S0, W0);
    evaluate_sample<KMAX, MT, FULL>(a, ray, z1, S1, W1);
    const float den = (S0 - S1) * (S0 - S1);
    const float gS[2] = {G * (z1 - z0) * (-S1) / den, G * (z1 - z0) * S0 / den};
    const MT *map = reinterpret_cast<const MT *>(a.dw);
    const size_t plane = (size_t)a.W * a.H;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float zs = t ? z1 : z0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (FULL || k < a.K) {
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

// Pass 1.  Only target pixels with a crossing (and a non-zero upstream
// gradient) have work, about a third of them on the 8 x 1080p frame; so each
// block of 128 threads first lists the pixels with work among its 16 x 32 tile
// (in raster order, through a block-wide prefix count of warp ballots) and then
// deals the list out to its threads, which keeps the warps full.  Its gathers
// and atomics wait on memory: twelve resident blocks per SM (40 registers, a few
// spilled) hide more of that than eight at 64 registers (130.8 -> 123.3 us).
// FULL: the call has exactly KMAX views (no per-view guard).
constexpr int BS_TX = 16, BS_TY = 32, BS_THREADS = 128;
template <int KMAX, typename MT, bool FULL>
__global__ void __launch_bounds__(BS_THREADS, 12) fuse_bwd_scatter(const FuseArgs a, const int16_t *__restrict__ crossing,
                                                               const float *__restrict__ grad_fused,
                                                               float2 *__restrict__ acc) {
    constexpr int PER = BS_TX * BS_TY / BS_THREADS;  // pixels per thread in the listing pass
    __shared__ int s_list[BS_TX * BS_TY];
    __shared__ int s_warp[BS_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int base = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int e = r * BS_THREADS + tid;  // tile-local raster index
        const int i = blockIdx.x * BS_TX + (e % BS_TX), j = blockIdx.y * BS_TY + (e / BS_TX);
        bool work = false;
        if (i < a.Wt && j < a.Ht) {
            const size_t o = (size_t)j * a.Wt + i;
            const int s = crossing[o];
            work = s >= 0 && s + 1 < a.D && grad_fused[o] != 0.0f;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, work);
        if (lane == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        int before = base;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        int total = base;
        for (int w = 0; w < BS_THREADS / 32; ++w) total += s_warp[w];
        if (work) s_list[before + __popc(ball & ((1u << lane) - 1u))] = e;
        __syncthreads();  // s_warp is rewritten by the next round
        base = total;
    }
    for (int q = tid; q < base; q += BS_THREADS) {
        const int e = s_list[q];
        const int i = blockIdx.x * BS_TX + (e % BS_TX), j = blockIdx.y * BS_TY + (e / BS_TX);
        const size_t o = (size_t)j * a.Wt + i;
        bwd_pixel<KMAX, MT, FULL>(a, i, j, crossing[o], grad_fused[o], acc);
    }
}

template <int KMAX, typename MT>
void bwd_scatter_k(const FuseArgs &a, const int16_t *crossing, const float *grad_fused, float2 *acc,
                   cudaStream_t st) {
    const dim3 grid((a.Wt + BS_TX - 1) / BS_TX, (a.Ht + BS_TY - 1) / BS_TY), block(BS_THREADS);
    if (a.K == KMAX) fuse_bwd_scatter<KMAX, MT, true><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
    else fuse_bwd_scatter<KMAX, MT, false><<<grid, block, 0, st>>>(a, crossing, grad_fused, acc);
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

#ifndef GVS_GATHER_ROWS
#define GVS_GATHER_ROWS 4  // 8 reads fewer shared values per output but runs fewer warps: 278 -> 312 us
#endif
constexpr int GB_TX = 32;                 // block of 32 x 32 input pixels: 32 x (32 / GB_ROWS) threads,
constexpr int GB_TY = 32;                 // each thread GB_ROWS consecutive rows
constexpr int GB_ROWS = GVS_GATHER_ROWS;
static_assert(GB_TY % GB_ROWS == 0, "the rows split evenly among the thread rows");

// P(c) = A(c) domega/dnu(c) at input pixel (cx, cy) of view k, or 0 outside the
// image, where A = 0, at an invalid centre (dc NaN) or where the weight is
// saturated.  dtc: the depth tile at c's window corner (re-sum of nu without a map).
template <int R, int DW>
__device__ __forceinline__ float adjoint_p(const float2 *__restrict__ ak, const float2 *__restrict__ wk, int cx,
                                           int cy, int W, int H, float dc, const float (*dtc)[DW], int ox, float mu,
                                           float wconst, float inv_w2) {
    float P = 0.0f;
    if (cx >= 0 && cx < W && cy >= 0 && cy < H) {
        const float A = ak[(size_t)cy * W + cx].x;
        if (A != 0.0f && dc == dc) {
            if (wk) {
                const float om = __ldg(&wk[(size_t)cy * W + cx]).y;
                if (om < 1.0f) P = A * (-0.5f * om * om * om * (inv_w2 / (wconst * wconst)));
            } else {
                float nu = 0.0f;
                for (int dy = 0; dy <= 2 * R; ++dy)
                    for (int dx = 0; dx <= 2 * R; ++dx) {
                        const float t = fminf(fabsf(dc - dtc[dy][ox + dx]), mu);
                        nu = fmaf(t, t, nu);
                    }
                const float unclamped = nu > 0.0f ? wconst * rsqrtf(nu * inv_w2) : 2.0f;
                if (unclamped < 1.0f) P = A * (-0.5f * unclamped / nu);
            }
        }
    }
    return P;
}

// wmap: the forward's float2 (d, omega) planes, or null (re-sum nu).
// The P tile holds 2 P(c): every term of the gradient carries the factor 2
// (d/dd (d - n)^2), and scaling by 2 is exact, so 2 (d_x - d_n)(P(x) + P(n))
// = (d_x - d_n)(2 P(x) + 2 P(n)) bit for bit with one multiplication fewer per
// term; the border path halves its own sums instead, again exactly.
template <int R, typename DT>
__global__ void __launch_bounds__(GB_TX *(GB_TY / GB_ROWS)) fuse_bwd_gather(const DT *__restrict__ depth,
                                                                const float2 *__restrict__ wmap,
                                                                const float2 *__restrict__ acc,
                                                                float *__restrict__ grad, int W, int H, float mu,
                                                                float wconst, float inv_w2) {
    constexpr int DW = GB_TX + 4 * R, DH = GB_TY + 4 * R;   // depths: outputs + 2R halo
    constexpr int PW = GB_TX + 2 * R, PH = GB_TY + 2 * R;   // 2 P(c): outputs + R halo
    constexpr int TR = GB_TY / GB_ROWS;                     // thread rows
    static_assert(DW - GB_TX <= GB_TX && PW - GB_TX <= GB_TX, "the halo columns fit one more pass of the lanes");
    __shared__ float dt[DH][DW];
    __shared__ float pt[PH][PW];
    const int k = blockIdx.z;
    const DT *dep = depth + (size_t)k * W * H;
    const float2 *ak = acc + (size_t)k * W * H;
    const float2 *wk = wmap ? wmap + (size_t)k * W * H : nullptr;
    const int bx = blockIdx.x * GB_TX, by = blockIdx.y * GB_TY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    {
        // depth tile by rows: each lane's two clamped columns computed once
        const int gxa = min(max(bx - 2 * R + tx, 0), W - 1);
        const int gxb = min(max(bx - 2 * R + GB_TX + tx, 0), W - 1);
        const bool has_b = tx < DW - GB_TX;
#pragma unroll 2
        for (int sy = ty; sy < DH; sy += TR) {
            const DT *row = dep + (size_t)min(max(by - 2 * R + sy, 0), H - 1) * W;
            const float da = load_depth(&row[gxa]);
            dt[sy][tx] = valid_depth(da) ? da : __int_as_float(0x7fc00000);  // NaN marks invalid
            if (has_b) {
                const float db = load_depth(&row[gxb]);
                dt[sy][GB_TX + tx] = valid_depth(db) ? db : __int_as_float(0x7fc00000);
            }
        }
    }
    __syncthreads();
    // 2 P(c) on the outputs and an R halo
#pragma unroll 1
    for (int py = ty; py < PH; py += TR) {
        const int cy = by - R + py;
        pt[py][tx] = 2.0f * adjoint_p<R, DW>(ak, wk, bx - R + tx, cy, W, H, dt[py + R][tx + R], dt + py, tx, mu,
                                             wconst, inv_w2);
        if (tx < PW - GB_TX)
            pt[py][GB_TX + tx] = 2.0f * adjoint_p<R, DW>(ak, wk, bx - R + GB_TX + tx, cy, W, H,
                                                         dt[py + R][GB_TX + tx + R], dt + py, GB_TX + tx, mu,
                                                         wconst, inv_w2);
    }
    __syncthreads();
    // a block whose windows of windows stay inside the image sees every window entry once
    const bool interior = bx >= 2 * R && by >= 2 * R && bx + GB_TX + 2 * R <= W && by + GB_TY + 2 * R <= H;
    const int x = bx + tx;
    const int ly0 = ty * GB_ROWS;  // this thread's GB_ROWS consecutive rows
    if (interior) {
        // entry n of x's window and window centre c = n coincide: one pass,
        // (d_x - d_n) (2 P(x) + 2 P(n)) where |d_x - d_n| < mu (false for an invalid n, and
        // for an invalid x, whose NaN depth fails every test).  The thread's outputs share
        // their window rows: each shared value is read once and serves every output whose
        // window holds it, each output taking its entries in the same order as alone.
        float dx0[GB_ROWS], Px2[GB_ROWS], g[GB_ROWS];
#pragma unroll
        for (int p = 0; p < GB_ROWS; ++p) {
            dx0[p] = dt[ly0 + p + 2 * R][tx + 2 * R];
            Px2[p] = pt[ly0 + p + R][tx + R];
            g[p] = ak[(size_t)(by + ly0 + p) * W + x].y;  // B(x)
        }
#pragma unroll
        for (int r = 0; r < GB_ROWS + 2 * R; ++r) {
#pragma unroll
            for (int ox = -R; ox <= R; ++ox) {
                const float dn = dt[ly0 + R + r][tx + 2 * R + ox];
                const float pn2 = pt[ly0 + r][tx + R + ox];
#pragma unroll
                for (int p = 0; p < GB_ROWS; ++p) {
                    if (r - p < 0 || r - p > 2 * R) continue;  // row offset oy = r - p - R outside the window
                    const float diff = dx0[p] - dn;
                    if (fabsf(diff) < mu) g[p] = fmaf(diff, Px2[p] + pn2, g[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < GB_ROWS; ++p) grad[(size_t)k * W * H + (size_t)(by + ly0 + p) * W + x] = g[p];
        return;
    }
#pragma unroll 1
    for (int rr = 0; rr < GB_ROWS; ++rr) {
        const int ly = ly0 + rr;  // row within the block
        const int y = by + ly;
        if (x >= W || y >= H) continue;
        const float dx0 = dt[ly + 2 * R][tx + 2 * R];
        float g = ak[(size_t)y * W + x].y;  // B(x)
        if (dx0 == dx0) {
            const float Px2 = pt[ly + R][tx + R];
            if (Px2 != 0.0f) {
                // P(x) sum 2 (d_x - d_n) = 2 P(x) sum (d_x - d_n): every partial sum halved exactly
                float sum = 0.0f;
                for (int ey = -R; ey <= R; ++ey)
                    for (int ex = -R; ex <= R; ++ex) {
                        const float dn = dt[ly + 2 * R + ey][tx + 2 * R + ex];
                        const float diff = dx0 - dn;
                        if (fabsf(diff) < mu) sum += diff;  // false for a NaN (invalid) neighbour
                    }
                g += Px2 * sum;
            }
            for (int cyo = -R; cyo <= R; ++cyo) {
                const int my = window_multiplicity(y + cyo, y, H, R);
                if (my == 0) continue;
                for (int cxo = -R; cxo <= R; ++cxo) {
                    const int mx = window_multiplicity(x + cxo, x, W, R);
                    if (mx == 0) continue;
                    const float Pc2 = pt[ly + R + cyo][tx + R + cxo];
                    if (Pc2 == 0.0f) continue;
                    const float diff = dt[ly + 2 * R + cyo][tx + 2 * R + cxo] - dx0;
                    // m P(c) (-2) diff = -(m 2 P(c)) diff
                    if (fabsf(diff) < mu) g += -((float)(mx * my) * Pc2) * diff;
                }
            }
        }
        grad[(size_t)k * W * H + (size_t)y * W + x] = g;
    }
}

template <int R, typename DT>
cudaError_t launch_bwd_gather_r(const void *depth, const float2 *wmap, const float2 *acc, float *grad, int K, int W,
                                int H, float mu, float wconst, float inv_w2, cudaStream_t st) {
    dim3 grid((W + GB_TX - 1) / GB_TX, (H + GB_TY - 1) / GB_TY, K);
    fuse_bwd_gather<R, DT><<<grid, dim3(GB_TX, GB_TY / GB_ROWS), 0, st>>>(reinterpret_cast<const DT *>(depth), wmap, acc, grad,
                                                                W, H, mu, wconst, inv_w2);
    return cudaGetLastError();
}

template <typename DT>
cudaError_t launch_bwd_gather(const void *depth, const float2 *wmap, const float2 *acc, float *grad, int K, int W,
                              int H, float mu, float wconst, int window, cudaStream_t st) {
    const float inv_w2 = (float)(1.0 / ((double)window * (double)window));
    switch (window / 2) {
        case 0: return launch_bwd_gather_r<0, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 1: return launch_bwd_gather_r<1, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 2: return launch_bwd_gather_r<2, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 3: return launch_bwd_gather_r<3, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 4: return launch_bwd_gather_r<4, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 5: return launch_bwd_gather_r<5, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 6: return launch_bwd_gather_r<6, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        case 7: return launch_bwd_gather_r<7, DT>(depth, wmap, acc, grad, K, W, H, mu, wconst, inv_w2, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fuse_backward(const FuseArgs &a, const void *depth, int depth_dtype, const int16_t *crossing,
                                 const float *grad_fused, float *grad_depths, float2 *acc, float mu, float wconst,
                                 int window, cudaStream_t st) {
    if (a.K == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)a.K * a.W * a.H * sizeof(float2), st);
    if (e != cudaSuccess) return e;
    if (a.map_dtype == GVS_F16) {
        if (a.K <= 4) bwd_scatter_k<4, __half2>(a, crossing, grad_fused, acc, st);
        else if (a.K <= 8) bwd_scatter_k<8, __half2>(a, crossing, grad_fused, acc, st);
        else if (a.K <= 16) bwd_scatter_k<16, __half2>(a, crossing, grad_fused, acc, st);
        else bwd_scatter_k<32, __half2>(a, crossing, grad_fused, acc, st);
    } else {
        if (a.K <= 4) bwd_scatter_k<4, float2>(a, crossing, grad_fused, acc, st);
        else if (a.K <= 8) bwd_scatter_k<8, float2>(a, crossing, grad_fused, acc, st);
        else if (a.K <= 16) bwd_scatter_k<16, float2>(a, crossing, grad_fused, acc, st);
        else bwd_scatter_k<32, float2>(a, crossing, grad_fused, acc, st);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float2 *wmap = a.map_dtype == GVS_F16 ? nullptr : reinterpret_cast<const float2 *>(a.dw);
    return depth_dtype == GVS_F16
               ? launch_bwd_gather<__half>(depth, wmap, acc, grad_depths, a.K, a.W, a.H, mu, wconst, window, st)
               : launch_bwd_gather<float>(depth, wmap, acc, grad_depths, a.K, a.W, a.H, mu, wconst, window, st);
}

GVS_BOUNDS_TAKE_FN(bounds_take_fuse_bwd)

}  // namespace gvs
