/*
 * FP64 CPU oracle for the geometry core of "Geometry-guided Online 3D Video
 * Synthesis with Multi-View Temporal Consistency" (arXiv 2505.18932).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this; it
 * exists so that the CUDA library can be checked against a plain, slow,
 * obviously-correct statement of what the method computes.  It shares no
 * code, header or table with the CUDA library.
 *
 * What it follows:
 *   refine     Sec. 3.2, Eq. 1 and Eq. 2 (temporal depth filtering), in the
 *              binary form: m = [max_c |I^t_c - I^{t-1}_c| > floor(255 tau)],
 *              D'^t = m ? D^t : D'^{t-1}; at t = 0, m = 1.
 *   weight     Supplement A.1 (confidence weight): nu = sum over the w x w
 *              window of min((D[c] - D[n])^2, tau^2); omega = min(0.001 *
 *              (nu / w^2)^(-1/2), 1).  Evaluated PER SAMPLE at the sampled
 *              pixel (no precomputed map).
 *   fuse       Supplement A.1 (projection, signed distance, weighted sum of
 *              clamped distances, omega = 0 behind the truncation band),
 *              Eq. 3 (raymarch), with D uniform samples and the first +/-
 *              zero crossing interpolated linearly.
 *   splat      Sec. 3.1 and Supplement A.3 (each input view forward-rendered
 *              separately with pixel-sized, fully opaque primitives, depth
 *              test for occlusion), as a z-buffer with a pixel footprint.
 *   gauss      the same render with pixel-sized isotropic 3D Gaussians,
 *              alpha-composited front to back by the rasterisation rules of
 *              3D Gaussian splatting (see orc_gauss_splat).
 *
 * Readings where the paper is silent or inconsistent:
 *   - sign: sdf = (d_in - z_proj) / mu, positive in front of the surface,
 *     omega = 0 where sdf < -1; the printed s_k = z_k - D_k would make free
 *     space negative, at odds with the "omega = 0 if s_k < -tau" rule and the
 *     forward stepping by 0.8 s.
 *   - D_k[u,v] samples the NEAREST pixel (ties to even); the window is
 *     clamped at image borders; a neighbour with invalid depth contributes
 *     mu^2; an invalid centre gives omega = 0; nu = 0 gives omega = 1.
 *   - out of image, behind the camera (z <= 1e-6) or invalid depth: the
 *     view contributes nothing at that sample.
 *   - the fused value is the plain weighted sum (normalize = 0) or S/W.
 *   - crossing: first s with W_s > 0, W_{s+1} > 0, S_s > 0, S_{s+1} <= 0.
 *
 * Precision: FP64 throughout, EXCEPT the decisions that turn floating point
 * into integers, which are taken in the GPU kernel's precision (FP32) by an
 * explicit address contract that both sides evaluate op for op:
 *   fuse : per-view FP32 matrix M, offset b (composed in FP64, rounded once),
 *          a = M [i j 1]^T by fused multiply-adds, sample z_s = fma(s, dz, zn),
 *          h = fma(z_s, a, b); the sampled pixel is the nearest integer to the
 *          exact quotients h.x/h.z, h.y/h.z.  The sample point is the FP32 z_s
 *          and the projected depth is h.z; everything after is FP64.
 *   splat: per-view FP32 A, c, f_ratio; m = A [u v 1]^T, h = fma(d, m, c),
 *          x = h.x/h.z, y = h.y/h.z rounded to FP32; footprint half-width
 *          hw = min(max(0.5 f_ratio (d/h.z), 0.5), max_hw); covered target
 *          pixels [ceil(x-hw), floor(x+hw)]; key (bits(z) << 32 | source).
 * Compile with -ffp-contract=off so that no other expression is fused.
 *
 * Parity pins live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double R[9];
    double t[3];
} orc_camera;

static int depth_valid(float d) { return isfinite(d) && d > 0.0f; }

/* ------------------------------------------------------------------------ */
/* Eq. 1 / Eq. 2 in the binary-mask form.                                   */
/* ------------------------------------------------------------------------ */
int orc_refine_depth(int n_views, int H, int W, const uint8_t *rgba_t, const uint8_t *rgba_prev,
                     const float *depth_t, const float *state_prev, float tau,
                     float *state_out, uint8_t *mask_out) {
    if (n_views <= 0 || H <= 0 || W <= 0 || !rgba_t || !depth_t || !state_out) return -1;
    int T = (int)floor(255.0 * (double)tau);
    size_t n = (size_t)n_views * H * W;
    for (size_t p = 0; p < n; ++p) {
        int m = 1;
        if (rgba_prev) {
            int dmax = 0;
            for (int c = 0; c < 3; ++c) {
                int d = abs((int)rgba_t[4 * p + c] - (int)rgba_prev[4 * p + c]);
                if (d > dmax) dmax = d;
            }
            m = dmax > T;
        }
        if (mask_out) mask_out[p] = (uint8_t)m;
        state_out[p] = (m || !rgba_prev || !state_prev) ? depth_t[p] : state_prev[p];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Supplement A.1: confidence weight of view k at pixel (u, v).             */
/* ------------------------------------------------------------------------ */
double orc_weight(const float *depth, int H, int W, int u, int v, double mu, double wconst, int window) {
    float dc = depth[(size_t)v * W + u];
    if (!depth_valid(dc)) return 0.0;
    int r = window / 2;
    double nu = 0.0;
    for (int dy = -r; dy <= r; ++dy) {
        for (int dx = -r; dx <= r; ++dx) {
            int q = v + dy, p = u + dx;
            q = q < 0 ? 0 : (q >= H ? H - 1 : q);
            p = p < 0 ? 0 : (p >= W ? W - 1 : p);
            float dn = depth[(size_t)q * W + p];
            if (!depth_valid(dn)) { nu += mu * mu; continue; }
            double diff = (double)dc - (double)dn;
            double sq = diff * diff;
            nu += sq < mu * mu ? sq : mu * mu;
        }
    }
    if (nu == 0.0) return 1.0;
    double w = wconst * pow(nu / (double)(window * window), -0.5);
    return w < 1.0 ? w : 1.0;
}

/* ------------------------------------------------------------------------ */
/* FP64 composition of the per-view FP32 contract coefficients.             */
/* Maps depth * [i j 1] in camera `from` to homogeneous pixel coordinates in */
/* camera `to`:  h = depth * (M [i j 1]^T) + b, with                         */
/* M = K_to R_to R_from^T K_from^-1 and b = K_to (t_to - R_to R_from^T t_from). */
/* ------------------------------------------------------------------------ */
static void compose(const orc_camera *to, const orc_camera *from, float M[9], float b[3]) {
    double Q[9], g[3], N[9], bb[3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Q[3 * r + c] = to->R[3 * r + 0] * from->R[3 * c + 0] + to->R[3 * r + 1] * from->R[3 * c + 1] +
                           to->R[3 * r + 2] * from->R[3 * c + 2];
    for (int r = 0; r < 3; ++r)
        g[r] = to->t[r] - (Q[3 * r + 0] * from->t[0] + Q[3 * r + 1] * from->t[1] + Q[3 * r + 2] * from->t[2]);
    for (int c = 0; c < 3; ++c) {
        N[0 + c] = to->fx * Q[0 + c] + to->cx * Q[6 + c];
        N[3 + c] = to->fy * Q[3 + c] + to->cy * Q[6 + c];
        N[6 + c] = Q[6 + c];
    }
    bb[0] = to->fx * g[0] + to->cx * g[2];
    bb[1] = to->fy * g[1] + to->cy * g[2];
    bb[2] = g[2];
    for (int r = 0; r < 3; ++r) {
        M[3 * r + 0] = (float)(N[3 * r + 0] / from->fx);
        M[3 * r + 1] = (float)(N[3 * r + 1] / from->fy);
        M[3 * r + 2] = (float)((N[3 * r + 2] - (N[3 * r + 0] * from->cx) / from->fx) - (N[3 * r + 1] * from->cy) / from->fy);
        b[r] = (float)bb[r];
    }
}

/* nearest integer (ties to even) of the exact real quotient num/den, den > 0 */
static double nearest_of_quotient(float num, float den) {
    return nearbyint((double)num / (double)den);
}

/* FP64 geometry of the same sample, used only for the informational count of
 * address decisions where FP32 and FP64 disagree. */
static void project_fp64(const orc_camera *view, const orc_camera *tgt, double i, double j, double z,
                         double *x, double *y, double *zk) {
    double P[3] = {z * (i - tgt->cx) / tgt->fx, z * (j - tgt->cy) / tgt->fy, z};
    double pw[3];
    for (int a = 0; a < 3; ++a)
        pw[a] = tgt->R[0 * 3 + a] * (P[0] - tgt->t[0]) + tgt->R[1 * 3 + a] * (P[1] - tgt->t[1]) +
                tgt->R[2 * 3 + a] * (P[2] - tgt->t[2]);
    double pc[3];
    for (int a = 0; a < 3; ++a)
        pc[a] = view->R[3 * a + 0] * pw[0] + view->R[3 * a + 1] * pw[1] + view->R[3 * a + 2] * pw[2] + view->t[a];
    *zk = pc[2];
    *x = (view->fx * pc[0] + view->cx * pc[2]) / pc[2];
    *y = (view->fy * pc[1] + view->cy * pc[2]) / pc[2];
}

typedef struct {
    const orc_camera *in_cams; const float *depths; int n_views;
    const orc_camera *target;
    int D; double z_near, z_far, mu, wconst; int window, normalize;
    const int32_t *pixels; int64_t n_pixels;
    double *out_depth; int32_t *out_index; uint8_t *out_amb;
    int64_t *addr_fp64_mismatch;
    float (*M)[9]; float (*b)[3];
    int64_t p0, p1;
    /* temporal term (Supplement A.2), per target pixel, or NULL */
    const float *tmp_depth, *tmp_weight;
    double *out_wview;
} fuse_job;

/* One target pixel: Supplement A.1 + Eq. 3 with D uniform samples. */
static void fuse_pixel(const fuse_job *jb, int i, int j, double *out_d, int32_t *out_s, uint8_t *out_a,
                       int64_t *mism) {
    const int K = jb->n_views;
    const int D = jb->D;
    const float zn = (float)jb->z_near;
    const float dz = (float)((jb->z_far - jb->z_near) / (double)(D - 1));
    const double mu = jb->mu;
    int amb = 0;
    double S_prev = 0.0, W_prev = 0.0, z_prev = 0.0, Wv_prev = 0.0;
    double td = 0.0, tw = 0.0;
    if (jb->tmp_depth) {
        size_t tp = (size_t)j * jb->target->width + i;
        if (depth_valid(jb->tmp_depth[tp]) && jb->tmp_weight[tp] > 0.0f) {
            td = jb->tmp_depth[tp];
            tw = jb->tmp_weight[tp];
        }
    }
    if (jb->out_wview) jb->out_wview[(size_t)j * jb->target->width + i] = 0.0;
    *out_d = 0.0;
    *out_s = -1;
    for (int s = 0; s < D; ++s) {
        float zs = fmaf((float)s, dz, zn);
        double S = 0.0, Wt = 0.0;
        for (int k = 0; k < K; ++k) {
            const orc_camera *vc = &jb->in_cams[k];
            const float *M = jb->M[k];
            const float *b = jb->b[k];
            float a0 = fmaf(M[0], (float)i, fmaf(M[1], (float)j, M[2]));
            float a1 = fmaf(M[3], (float)i, fmaf(M[4], (float)j, M[5]));
            float a2 = fmaf(M[6], (float)i, fmaf(M[7], (float)j, M[8]));
            float h0 = fmaf(zs, a0, b[0]);
            float h1 = fmaf(zs, a1, b[1]);
            float h2 = fmaf(zs, a2, b[2]);
            if (!(h2 > 1e-6f)) continue;
            double u = nearest_of_quotient(h0, h2);
            double v = nearest_of_quotient(h1, h2);
            if (mism) {
                double x64, y64, z64;
                project_fp64(vc, jb->target, i, j, (double)zs, &x64, &y64, &z64);
                if (nearbyint(x64) != u || nearbyint(y64) != v) ++*mism;
            }
            if (u < 0 || v < 0 || u > vc->width - 1 || v > vc->height - 1) continue;
            const float *dep = jb->depths + (size_t)k * vc->width * vc->height;
            float d = dep[(size_t)v * vc->width + (size_t)u];
            if (!depth_valid(d)) continue;
            double sdf = ((double)d - (double)h2) / mu;
            if (fabs(sdf + 1.0) < 1e-5) amb = 1;
            if (sdf < -1.0) continue; /* hidden behind the truncation band */
            double w = orc_weight(dep, vc->height, vc->width, (int)u, (int)v, mu, jb->wconst, jb->window);
            double c = sdf < -1.0 ? -1.0 : (sdf > 1.0 ? 1.0 : sdf);
            S += w * c;
            Wt += w;
        }
        double Wv = Wt; /* the input views' weight, before the temporal term */
        if (tw > 0.0) {
            /* Supplement A.2: the previous output depth as one more TSDF input, at the same pixel */
            double sdf = (td - (double)zs) / mu;
            if (fabs(sdf + 1.0) < 1e-5) amb = 1;
            if (sdf >= -1.0) {
                S += tw * (sdf > 1.0 ? 1.0 : sdf);
                Wt += tw;
            }
        }
        if (jb->normalize && Wt > 0.0) S /= Wt;
        double scale = jb->normalize ? 1.0 : Wt;
        if (Wt > 0.0 && fabs(S) <= 1e-5 * scale) amb = 1;
        if (s > 0 && W_prev > 0.0 && Wt > 0.0 && S_prev > 0.0 && S <= 0.0) {
            double t = S_prev / (S_prev - S);
            *out_d = z_prev + ((double)zs - z_prev) * t;
            *out_s = s - 1;
            /* conditioning of the interpolation against FP32 rounding of S */
            double sens = ((double)zs - z_prev) * 1e-5 * (jb->normalize ? 2.0 : (W_prev + Wt)) / (S_prev - S);
            if (sens > 0.25e-4 * fabs(*out_d)) amb = 1;
            if (jb->out_wview) jb->out_wview[(size_t)j * jb->target->width + i] = Wv_prev + t * (Wv - Wv_prev);
            break;
        }
        S_prev = S;
        W_prev = Wt;
        Wv_prev = Wv;
        z_prev = (double)zs;
    }
    *out_a = (uint8_t)amb;
}

static void *fuse_worker(void *arg) {
    fuse_job *jb = (fuse_job *)arg;
    int Wt = jb->target->width;
    for (int64_t p = jb->p0; p < jb->p1; ++p) {
        int i, j;
        if (jb->pixels) { i = jb->pixels[2 * p]; j = jb->pixels[2 * p + 1]; }
        else { i = (int)(p % Wt); j = (int)(p / Wt); }
        uint8_t a;
        fuse_pixel(jb, i, j, &jb->out_depth[p], &jb->out_index[p], &a, jb->addr_fp64_mismatch);
        if (jb->out_amb) jb->out_amb[p] = a;
    }
    return NULL;
}

int orc_fuse_depth(const orc_camera *in_cams, const float *depths, int n_views, const orc_camera *target,
                   int num_samples, double z_near, double z_far, double mu, double weight_const, int window,
                   int normalize, const int32_t *pixels, int64_t n_pixels,
                   double *out_depth, int32_t *out_index, uint8_t *out_amb, int64_t *addr_fp64_mismatch,
                   int n_threads) {
    if (!in_cams || !depths || n_views <= 0 || !target || num_samples < 2 || !(z_near < z_far) || !(mu > 0) ||
        window < 1 || !out_depth || !out_index)
        return -1;
    if (!pixels) n_pixels = (int64_t)target->width * target->height;
    float (*M)[9] = malloc(sizeof(float[9]) * n_views);
    float (*b)[3] = malloc(sizeof(float[3]) * n_views);
    for (int k = 0; k < n_views; ++k) compose(&in_cams[k], target, M[k], b[k]);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    int64_t mism[256];
    fuse_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) {
        mism[t] = 0;
        fuse_job jb = {in_cams, depths, n_views, target, num_samples, z_near, z_far, mu, weight_const, window,
                       normalize, pixels, n_pixels, out_depth, out_index, out_amb,
                       addr_fp64_mismatch ? &mism[t] : NULL, M, b,
                       n_pixels * t / n_threads, n_pixels * (t + 1) / n_threads, NULL, NULL, NULL};
        jobs[t] = jb;
    }
    int started = 0;
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, fuse_worker, &jobs[t]) != 0) break;
        started = t;
    }
    fuse_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < n_threads; ++t) fuse_worker(&jobs[t]);
    if (addr_fp64_mismatch) {
        int64_t tot = 0;
        for (int t = 0; t < n_threads; ++t) tot += mism[t];
        *addr_fp64_mismatch = tot;
    }
    free(M);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 / Supplement A.3: per-view forward render with a depth test.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ok;
    float x, y, z;
    int i0, i1, j0, j1; /* covered target pixels, inclusive, clipped */
} splat_geo;

static splat_geo splat_contract(const float A[9], const float c[3], float f_ratio, int footprint, float max_hw,
                                int u, int v, float d, int Wt, int Ht) {
    splat_geo g = {0};
    if (!depth_valid(d)) return g;
    float m0 = fmaf(A[0], (float)u, fmaf(A[1], (float)v, A[2]));
    float m1 = fmaf(A[3], (float)u, fmaf(A[4], (float)v, A[5]));
    float m2 = fmaf(A[6], (float)u, fmaf(A[7], (float)v, A[8]));
    float h0 = fmaf(d, m0, c[0]);
    float h1 = fmaf(d, m1, c[1]);
    float h2 = fmaf(d, m2, c[2]);
    if (!(h2 > 1e-6f)) return g;
    float x = h0 / h2, y = h1 / h2;
    float lo_x, hi_x, lo_y, hi_y;
    if (footprint) {
        float rho = f_ratio * (d / h2);
        float hw = 0.5f * rho;
        hw = hw > 0.5f ? hw : 0.5f;
        hw = hw < max_hw ? hw : max_hw;
        lo_x = ceilf(x - hw); hi_x = floorf(x + hw);
        lo_y = ceilf(y - hw); hi_y = floorf(y + hw);
    } else {
        lo_x = hi_x = rintf(x);
        lo_y = hi_y = rintf(y);
    }
    if (lo_x < 0.0f) lo_x = 0.0f;
    if (lo_y < 0.0f) lo_y = 0.0f;
    if (hi_x > (float)(Wt - 1)) hi_x = (float)(Wt - 1);
    if (hi_y > (float)(Ht - 1)) hi_y = (float)(Ht - 1);
    if (!(lo_x <= hi_x) || !(lo_y <= hi_y)) return g;
    g.ok = 1; g.x = x; g.y = y; g.z = h2;
    g.i0 = (int)lo_x; g.i1 = (int)hi_x; g.j0 = (int)lo_y; g.j1 = (int)hi_y;
    return g;
}

static uint64_t make_key(float z, uint32_t src) {
    uint32_t zb;
    memcpy(&zb, &z, 4);
    return ((uint64_t)zb << 32) | (uint64_t)src;
}

int orc_forward_splat(const orc_camera *in_cams, const float *depths, const uint32_t *rgba, int n_views,
                      const orc_camera *target, int footprint, float max_hw, float mu_guide, int guide_reject,
                      const double *fused, int32_t *winner, uint32_t *warped_rgba, float *warped_depth,
                      uint8_t *alpha, uint8_t *guided, uint8_t *guided_amb, int64_t *fp64_mismatch) {
    if (!in_cams || !depths || !rgba || n_views <= 0 || !target || !winner) return -1;
    if (guide_reject && !fused) return -1;
    int Wt = target->width, Ht = target->height;
    size_t np = (size_t)Wt * Ht;
    uint64_t *key = malloc(sizeof(uint64_t) * np);
    double *zb64 = fp64_mismatch ? malloc(sizeof(double) * np) : NULL;
    int64_t *src64 = fp64_mismatch ? malloc(sizeof(int64_t) * np) : NULL;
    if (fp64_mismatch) *fp64_mismatch = 0;
    size_t in_off = 0;
    for (int k = 0; k < n_views; ++k) {
        const orc_camera *vc = &in_cams[k];
        int W = vc->width, H = vc->height;
        float A[9], c[3];
        compose(target, vc, A, c);
        float f_ratio = (float)(target->fx / vc->fx);
        for (size_t p = 0; p < np; ++p) key[p] = ~(uint64_t)0;
        for (int v = 0; v < H; ++v) {
            for (int u = 0; u < W; ++u) {
                float d = depths[in_off + (size_t)v * W + u];
                splat_geo g = splat_contract(A, c, f_ratio, footprint, max_hw, u, v, d, Wt, Ht);
                if (!g.ok) continue;
                uint64_t kk = make_key(g.z, (uint32_t)(v * W + u));
                for (int jj = g.j0; jj <= g.j1; ++jj)
                    for (int ii = g.i0; ii <= g.i1; ++ii) {
                        if (guide_reject) {
                            /* the alternative reading of the fused-depth guidance (Sec. 3.1): a candidate
                             * in front of the fused surface by more than mu takes no part in the depth
                             * test; an integer decision, taken in FP32 like the kernel's */
                            float lim = (float)fused[(size_t)jj * Wt + ii] - mu_guide;
                            if (g.z < lim) continue;
                        }
                        uint64_t *slot = &key[(size_t)jj * Wt + ii];
                        if (kk < *slot) *slot = kk;
                    }
            }
        }
        if (fp64_mismatch) {
            /* same rule with FP64 geometry; informational only */
            for (size_t p = 0; p < np; ++p) { zb64[p] = INFINITY; src64[p] = -1; }
            for (int v = 0; v < H; ++v) {
                for (int u = 0; u < W; ++u) {
                    float d = depths[in_off + (size_t)v * W + u];
                    if (!depth_valid(d)) continue;
                    double x, y, z;
                    project_fp64(target, vc, u, v, d, &x, &y, &z);
                    if (!(z > 1e-6)) continue;
                    double lx, hx, ly, hy;
                    if (footprint) {
                        double hw = 0.5 * (target->fx / vc->fx) * ((double)d / z);
                        hw = hw > 0.5 ? hw : 0.5;
                        hw = hw < max_hw ? hw : max_hw;
                        lx = ceil(x - hw); hx = floor(x + hw); ly = ceil(y - hw); hy = floor(y + hw);
                    } else {
                        lx = hx = nearbyint(x); ly = hy = nearbyint(y);
                    }
                    if (lx < 0) lx = 0;
                    if (ly < 0) ly = 0;
                    if (hx > Wt - 1) hx = Wt - 1;
                    if (hy > Ht - 1) hy = Ht - 1;
                    for (double jj = ly; jj <= hy; jj += 1.0)
                        for (double ii = lx; ii <= hx; ii += 1.0) {
                            size_t q = (size_t)jj * Wt + (size_t)ii;
                            int64_t s = (int64_t)v * W + u;
                            if (z < zb64[q] || (z == zb64[q] && s < src64[q])) { zb64[q] = z; src64[q] = s; }
                        }
                }
            }
        }
        for (size_t p = 0; p < np; ++p) {
            size_t o = (size_t)k * np + p;
            uint64_t kk = key[p];
            int has = kk != ~(uint64_t)0;
            int32_t w = has ? (int32_t)(uint32_t)(kk & 0xffffffffu) : -1;
            uint32_t zb = (uint32_t)(kk >> 32);
            float z;
            memcpy(&z, &zb, 4);
            if (!has) z = 0.0f;
            winner[o] = w;
            if (warped_rgba) warped_rgba[o] = has ? rgba[in_off + (size_t)w] : 0u;
            if (warped_depth) warped_depth[o] = z;
            if (alpha) alpha[o] = (uint8_t)has;
            if (guided) {
                int gk = 0, ga = 0;
                if (has && fused) {
                    double diff = fabs((double)z - fused[p]) - (double)mu_guide;
                    gk = diff <= 0.0;
                    ga = fabs(diff) <= 1e-4 * fabs(fused[p]) + 1e-6;
                }
                guided[o] = (uint8_t)gk;
                if (guided_amb) guided_amb[o] = (uint8_t)ga;
            }
            if (fp64_mismatch && (int64_t)w != src64[p]) ++*fp64_mismatch;
        }
        in_off += (size_t)W * H;
    }
    free(key);
    free(zb64);
    free(src64);
    return 0;
}

/* Brute force of the same rule, target-major: for every target pixel scan
 * every source pixel.  Used on tiny images to check the scatter bookkeeping. */
int orc_splat_bruteforce(const orc_camera *in_cams, const float *depths, int n_views, const orc_camera *target,
                         int footprint, float max_hw, int32_t *winner) {
    int Wt = target->width, Ht = target->height;
    size_t in_off = 0;
    for (int k = 0; k < n_views; ++k) {
        const orc_camera *vc = &in_cams[k];
        int W = vc->width, H = vc->height;
        float A[9], c[3];
        compose(target, vc, A, c);
        float f_ratio = (float)(target->fx / vc->fx);
        for (int jj = 0; jj < Ht; ++jj)
            for (int ii = 0; ii < Wt; ++ii) {
                uint64_t best = ~(uint64_t)0;
                for (int v = 0; v < H; ++v)
                    for (int u = 0; u < W; ++u) {
                        float d = depths[in_off + (size_t)v * W + u];
                        splat_geo g = splat_contract(A, c, f_ratio, footprint, max_hw, u, v, d, Wt, Ht);
                        if (!g.ok || ii < g.i0 || ii > g.i1 || jj < g.j0 || jj > g.j1) continue;
                        uint64_t kk = make_key(g.z, (uint32_t)(v * W + u));
                        if (kk < best) best = kk;
                    }
                winner[(size_t)k * Wt * Ht + (size_t)jj * Wt + ii] =
                    best == ~(uint64_t)0 ? -1 : (int32_t)(uint32_t)(best & 0xffffffffu);
            }
        in_off += (size_t)W * H;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the fused depth with respect to the input depths              */
/* (Supplement A.1 and Eq. 3 differentiated; normalize = 0).                */
/*                                                                          */
/* D = z_s + (z_{s+1} - z_s) S_s / (S_s - S_{s+1}) depends on the inputs    */
/* only through S_s and S_{s+1}.  For each view contributing at either      */
/* bracketing sample, with c = clamp(sdf, -1, 1) and omega the weight at the */
/* sampled pixel, S = sum omega c gives                                      */
/*   dS/dD(centre) = omega [ -1 < sdf < 1 ] / mu + c domega/dD(centre)       */
/*   dS/dD(n)      = c domega/dD(n)   for every window entry n               */
/* with domega/dnu = -0.5 weight_const w nu^(-3/2) when omega < 1 (0 when    */
/* saturated), dnu/dD(centre) = sum 2 (D_c - D_n) [ (D_c - D_n)^2 < mu^2 ]   */
/* and dnu/dD(n) = -2 (D_c - D_n) [ ... ] per entry (invalid neighbours add  */
/* the constant mu^2).  Clamp, cut-off, crossing index and the nearest-pixel */
/* choice are piecewise constant: no gradient (subgradient 0 at the kinks).  */
/* The scatter below is written per window entry, literally.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int contributes;
    int u, v;
    double sdf, c, w;
} orc_view_sample;

static void sample_detail(const fuse_job *jb, int i, int j, int s, orc_view_sample *vs, double *S_out) {
    const float zn = (float)jb->z_near;
    const float dz = (float)((jb->z_far - jb->z_near) / (double)(jb->D - 1));
    float zs = fmaf((float)s, dz, zn);
    double S = 0.0;
    for (int k = 0; k < jb->n_views; ++k) {
        const orc_camera *vc = &jb->in_cams[k];
        const float *M = jb->M[k];
        const float *b = jb->b[k];
        vs[k].contributes = 0;
        float a0 = fmaf(M[0], (float)i, fmaf(M[1], (float)j, M[2]));
        float a1 = fmaf(M[3], (float)i, fmaf(M[4], (float)j, M[5]));
        float a2 = fmaf(M[6], (float)i, fmaf(M[7], (float)j, M[8]));
        float h0 = fmaf(zs, a0, b[0]), h1 = fmaf(zs, a1, b[1]), h2 = fmaf(zs, a2, b[2]);
        if (!(h2 > 1e-6f)) continue;
        double u = nearest_of_quotient(h0, h2), v = nearest_of_quotient(h1, h2);
        if (u < 0 || v < 0 || u > vc->width - 1 || v > vc->height - 1) continue;
        const float *dep = jb->depths + (size_t)k * vc->width * vc->height;
        float d = dep[(size_t)v * vc->width + (size_t)u];
        if (!depth_valid(d)) continue;
        double sdf = ((double)d - (double)h2) / jb->mu;
        if (sdf < -1.0) continue;
        vs[k].contributes = 1;
        vs[k].u = (int)u;
        vs[k].v = (int)v;
        vs[k].sdf = sdf;
        vs[k].c = sdf > 1.0 ? 1.0 : sdf;
        vs[k].w = orc_weight(dep, vc->height, vc->width, (int)u, (int)v, jb->mu, jb->wconst, jb->window);
        S += vs[k].w * vs[k].c;
    }
    *S_out = S;
}

/* d omega / d D for one view's sampled pixel, scattered into grad (scaled by g). */
static void scatter_weight_grad(const float *dep, int H, int W, int u, int v, double mu, double wconst, int window,
                                double g, double *grad) {
    float dc = dep[(size_t)v * W + u];
    if (!depth_valid(dc)) return;
    int r = window / 2;
    double nu = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            int q = v + dy, p = u + dx;
            q = q < 0 ? 0 : (q >= H ? H - 1 : q);
            p = p < 0 ? 0 : (p >= W ? W - 1 : p);
            float dn = dep[(size_t)q * W + p];
            if (!depth_valid(dn)) { nu += mu * mu; continue; }
            double diff = (double)dc - (double)dn;
            nu += diff * diff < mu * mu ? diff * diff : mu * mu;
        }
    if (nu == 0.0) return;
    double unclamped = wconst * pow(nu / (double)(window * window), -0.5);
    if (unclamped >= 1.0) return; /* saturated weight: no gradient */
    double dw_dnu = -0.5 * unclamped / nu;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            int q = v + dy, p = u + dx;
            q = q < 0 ? 0 : (q >= H ? H - 1 : q);
            p = p < 0 ? 0 : (p >= W ? W - 1 : p);
            float dn = dep[(size_t)q * W + p];
            if (!depth_valid(dn)) continue;
            double diff = (double)dc - (double)dn;
            if (!(diff * diff < mu * mu)) continue;
            grad[(size_t)v * W + u] += g * dw_dnu * 2.0 * diff;
            grad[(size_t)q * W + p] -= g * dw_dnu * 2.0 * diff;
        }
}

int orc_fuse_depth_grad(const orc_camera *in_cams, const float *depths, int n_views, const orc_camera *target,
                        int num_samples, double z_near, double z_far, double mu, double weight_const, int window,
                        const double *grad_fused, double *grad_depths) {
    if (!in_cams || !depths || n_views <= 0 || n_views > 256 || !target || num_samples < 2 || !(z_near < z_far) ||
        !(mu > 0) || window < 1 || !grad_fused || !grad_depths)
        return -1;
    float (*M)[9] = malloc(sizeof(float[9]) * n_views);
    float (*b)[3] = malloc(sizeof(float[3]) * n_views);
    for (int k = 0; k < n_views; ++k) compose(&in_cams[k], target, M[k], b[k]);
    fuse_job jb = {in_cams, depths, n_views, target, num_samples, z_near, z_far, mu, weight_const, window,
                   0, NULL, 0, NULL, NULL, NULL, NULL, M, b, 0, 0, NULL, NULL, NULL};
    const int W = in_cams[0].width, H = in_cams[0].height;
    const size_t plane = (size_t)W * H;
    for (size_t q = 0; q < plane * n_views; ++q) grad_depths[q] = 0.0;
    orc_view_sample vs0[256], vs1[256];
    const float zn = (float)z_near;
    const float dz = (float)((z_far - z_near) / (double)(num_samples - 1));
    for (int j = 0; j < target->height; ++j)
        for (int i = 0; i < target->width; ++i) {
            double G = grad_fused[(size_t)j * target->width + i];
            if (G == 0.0) continue;
            double d_out;
            int32_t s;
            uint8_t amb;
            fuse_pixel(&jb, i, j, &d_out, &s, &amb, NULL);
            if (s < 0) continue;
            double S0, S1;
            sample_detail(&jb, i, j, s, vs0, &S0);
            sample_detail(&jb, i, j, s + 1, vs1, &S1);
            double z0 = (double)fmaf((float)s, dz, zn), z1 = (double)fmaf((float)(s + 1), dz, zn);
            double den = (S0 - S1) * (S0 - S1);
            double gS[2] = {G * (z1 - z0) * (-S1) / den, G * (z1 - z0) * S0 / den};
            for (int t = 0; t < 2; ++t) {
                orc_view_sample *vs = t ? vs1 : vs0;
                for (int k = 0; k < n_views; ++k) {
                    if (!vs[k].contributes) continue;
                    const float *dep = depths + (size_t)k * plane;
                    double *gk = grad_depths + (size_t)k * plane;
                    if (vs[k].sdf > -1.0 && vs[k].sdf < 1.0) gk[(size_t)vs[k].v * W + vs[k].u] += gS[t] * vs[k].w / mu;
                    scatter_weight_grad(dep, H, W, vs[k].u, vs[k].v, mu, weight_const, window, gS[t] * vs[k].c, gk);
                }
            }
        }
    free(M);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Differentiable colour splat (reading of Sec. 3.1 / Supplement A.3 with   */
/* the pixel-sized Gaussians kept as weights).  Per view and target pixel p: */
/* z_w = depth of the z-buffer winner (as in orc_forward_splat); the front  */
/* band S(p) = { covering sources q : z_q <= z_w + mu_band } (FP32 test, as  */
/* the kernel takes it); g_q = exp(-|(x_q, y_q) - p|^2 / (2 sigma_q^2)),      */
/* sigma_q = hw_q / 2 (the footprint half-width); colour                     */
/* I(p) = sum_S g_q c_q / sum_S g_q; warped depth z_w.  Colours are          */
/* [N][H][W][4] (the 4th channel is carried, not splatted).                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ok;
    float x, y, z, hw;
    int i0, i1, j0, j1;
    float m2;
} soft_geo;

static soft_geo soft_contract(const float A[9], const float c[3], float f_ratio, float max_hw, int u, int v, float d,
                              int Wt, int Ht) {
    soft_geo s;
    memset(&s, 0, sizeof(s));
    splat_geo g = splat_contract(A, c, f_ratio, 1, max_hw, u, v, d, Wt, Ht);
    if (!g.ok) return s;
    s.ok = 1;
    s.x = g.x; s.y = g.y; s.z = g.z;
    s.i0 = g.i0; s.i1 = g.i1; s.j0 = g.j0; s.j1 = g.j1;
    float rho = f_ratio * (d / g.z);
    float hw = 0.5f * rho;
    hw = hw > 0.5f ? hw : 0.5f;
    hw = hw < max_hw ? hw : max_hw;
    s.hw = hw;
    s.m2 = fmaf(A[6], (float)u, fmaf(A[7], (float)v, A[8]));
    return s;
}

/* Forward; also returns per target pixel the winner, z_w and sum g for reuse. */
int orc_soft_splat(const orc_camera *in_cams, const float *depths, const double *colors, int n_views,
                   const orc_camera *target, float max_hw, float mu_band, int32_t *winner, double *out_color,
                   float *out_depth, double *out_wsum, uint8_t *out_alpha) {
    if (!in_cams || !depths || !colors || n_views <= 0 || !target || !winner || !out_color) return -1;
    int Wt = target->width, Ht = target->height;
    size_t np = (size_t)Wt * Ht;
    uint64_t *key = malloc(sizeof(uint64_t) * np);
    double *acc = malloc(sizeof(double) * 4 * np);
    size_t in_off = 0;
    for (int k = 0; k < n_views; ++k) {
        const orc_camera *vc = &in_cams[k];
        int W = vc->width, H = vc->height;
        float A[9], c[3];
        compose(target, vc, A, c);
        float f_ratio = (float)(target->fx / vc->fx);
        for (size_t p = 0; p < np; ++p) key[p] = ~(uint64_t)0;
        for (size_t p = 0; p < 4 * np; ++p) acc[p] = 0.0;
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                float d = depths[in_off + (size_t)v * W + u];
                soft_geo g = soft_contract(A, c, f_ratio, max_hw, u, v, d, Wt, Ht);
                if (!g.ok) continue;
                uint64_t kk = make_key(g.z, (uint32_t)(v * W + u));
                for (int jj = g.j0; jj <= g.j1; ++jj)
                    for (int ii = g.i0; ii <= g.i1; ++ii)
                        if (kk < key[(size_t)jj * Wt + ii]) key[(size_t)jj * Wt + ii] = kk;
            }
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                float d = depths[in_off + (size_t)v * W + u];
                soft_geo g = soft_contract(A, c, f_ratio, max_hw, u, v, d, Wt, Ht);
                if (!g.ok) continue;
                double sig = 0.5 * (double)g.hw;
                const double *col = colors + 4 * (in_off + (size_t)v * W + u);
                for (int jj = g.j0; jj <= g.j1; ++jj)
                    for (int ii = g.i0; ii <= g.i1; ++ii) {
                        size_t p = (size_t)jj * Wt + ii;
                        uint32_t zb = (uint32_t)(key[p] >> 32);
                        float zw;
                        memcpy(&zw, &zb, 4);
                        float lim = zw + mu_band; /* FP32 sum, as the kernel forms it */
                        if (!(g.z <= lim)) continue;
                        double dx = (double)g.x - ii, dy = (double)g.y - jj;
                        double w = exp(-(dx * dx + dy * dy) / (2.0 * sig * sig));
                        for (int ch = 0; ch < 3; ++ch) acc[4 * p + ch] += w * col[ch];
                        acc[4 * p + 3] += w;
                    }
            }
        for (size_t p = 0; p < np; ++p) {
            size_t o = (size_t)k * np + p;
            int has = key[p] != ~(uint64_t)0;
            uint32_t zb = (uint32_t)(key[p] >> 32);
            float zw;
            memcpy(&zw, &zb, 4);
            winner[o] = has ? (int32_t)(uint32_t)(key[p] & 0xffffffffu) : -1;
            if (out_depth) out_depth[o] = has ? zw : 0.0f;
            if (out_alpha) out_alpha[o] = (uint8_t)has;
            if (out_wsum) out_wsum[o] = acc[4 * p + 3];
            for (int ch = 0; ch < 4; ++ch)
                out_color[4 * o + ch] = (has && ch < 3 && acc[4 * p + 3] > 0.0) ? acc[4 * p + ch] / acc[4 * p + 3] : 0.0;
        }
        in_off += (size_t)W * H;
    }
    free(key);
    free(acc);
    return 0;
}

/* Adjoint: grad_color [N][Ht][Wt][4] (4th ignored), grad_depth [N][Ht][Wt] or NULL.
 * d I / d c_q = g_q / sum g;  d I / d g_q = (c_q - I) / sum g;
 * g_q depends on d_q through (x_q, y_q) and sigma_q (when hw is not clamped);
 * the warped depth z_w depends on the winner's depth through dz/dd = m_2.
 * Band membership, coverage and the winner are piecewise constant. */
int orc_soft_splat_grad(const orc_camera *in_cams, const float *depths, const double *colors, int n_views,
                        const orc_camera *target, float max_hw, float mu_band, const double *grad_color,
                        const double *grad_depth, double *grad_in_depth, double *grad_in_color) {
    int Wt = target->width, Ht = target->height;
    size_t np = (size_t)Wt * Ht;
    size_t nin = 0;
    for (int k = 0; k < n_views; ++k) nin += (size_t)in_cams[k].width * in_cams[k].height;
    int32_t *win = malloc(sizeof(int32_t) * np * n_views);
    double *col = malloc(sizeof(double) * 4 * np * n_views);
    float *zd = malloc(sizeof(float) * np * n_views);
    double *ws = malloc(sizeof(double) * np * n_views);
    int rc = orc_soft_splat(in_cams, depths, colors, n_views, target, max_hw, mu_band, win, col, zd, ws, NULL);
    if (rc) return rc;
    for (size_t q = 0; q < nin; ++q) grad_in_depth[q] = 0.0;
    for (size_t q = 0; q < 4 * nin; ++q) grad_in_color[q] = 0.0;
    size_t in_off = 0;
    for (int k = 0; k < n_views; ++k) {
        const orc_camera *vc = &in_cams[k];
        int W = vc->width, H = vc->height;
        float A[9], c[3];
        compose(target, vc, A, c);
        float f_ratio = (float)(target->fx / vc->fx);
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                size_t qi = in_off + (size_t)v * W + u;
                float d = depths[qi];
                soft_geo g = soft_contract(A, c, f_ratio, max_hw, u, v, d, Wt, Ht);
                if (!g.ok) continue;
                /* derivatives of the contract geometry with respect to d (FP64) */
                float m0 = fmaf(A[0], (float)u, fmaf(A[1], (float)v, A[2]));
                float m1 = fmaf(A[3], (float)u, fmaf(A[4], (float)v, A[5]));
                double h2 = (double)g.z;
                double dx_dd = ((double)m0 - (double)g.x * g.m2) / h2;
                double dy_dd = ((double)m1 - (double)g.y * g.m2) / h2;
                double rho = (double)f_ratio * ((double)d / h2);
                double dhw_dd = (0.5 * rho > 0.5 && 0.5 * rho < (double)max_hw)
                                    ? 0.5 * (double)f_ratio * (double)c[2] / (h2 * h2) : 0.0;
                double sig = 0.5 * (double)g.hw, dsig_dd = 0.5 * dhw_dd;
                for (int jj = g.j0; jj <= g.j1; ++jj)
                    for (int ii = g.i0; ii <= g.i1; ++ii) {
                        size_t o = (size_t)k * np + (size_t)jj * Wt + ii;
                        float lim = zd[o] + mu_band;
                        if (!(g.z <= lim)) continue;
                        double ex = (double)g.x - ii, ey = (double)g.y - jj;
                        double r2 = ex * ex + ey * ey;
                        double w = exp(-r2 / (2.0 * sig * sig));
                        double dw_dd = w * (-(ex * dx_dd + ey * dy_dd) / (sig * sig) + r2 * dsig_dd / (sig * sig * sig));
                        double sw = ws[o];
                        for (int ch = 0; ch < 3; ++ch) {
                            double G = grad_color[4 * o + ch];
                            grad_in_color[4 * qi + ch] += G * w / sw;
                            grad_in_depth[qi] += G * (colors[4 * qi + ch] - col[4 * o + ch]) / sw * dw_dd;
                        }
                        if (grad_depth && win[o] == (int32_t)(v * W + u)) grad_in_depth[qi] += grad_depth[o] * (double)g.m2;
                    }
            }
        in_off += (size_t)W * H;
    }
    free(win); free(col); free(zd); free(ws);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 and Eq. 2 in the paper's soft form (Sec. 3.2):                      */
/*   M = min(|I^t - I^{t-1}| / lambda_t + beta, 1)  (beta 0.6, lambda_t 0.7) */
/* computed at quarter resolution, 3x3 max-pooled and bilinearly upsampled,  */
/*   D'^t = M D^t + (1 - M) D'^{t-1}.                                        */
/* Readings: |I^t - I^{t-1}| per pixel is the largest of the three channel   */
/* differences in [0, 1] (value / 255); the quarter-resolution value is the  */
/* mean over the 4x4 block (partial blocks at the right/bottom edge average  */
/* the pixels they have); the pooling window is clamped at the borders; the  */
/* upsampling samples the quarter grid at ((x + 0.5) / 4 - 0.5, ...) with    */
/* clamp-to-edge.  An invalid previous depth takes the new depth; an invalid */
/* new depth keeps the previous one.                                         */
/* ------------------------------------------------------------------------ */
int orc_refine_depth_soft(int n_views, int H, int W, const uint8_t *rgba_t, const uint8_t *rgba_prev,
                          const float *depth_t, const float *state_prev, double beta, double lambda_t,
                          double *state_out, double *mask_out) {
    if (n_views <= 0 || H <= 0 || W <= 0 || !rgba_t || !rgba_prev || !depth_t || !state_prev || !state_out) return -1;
    int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    double *mq = malloc(sizeof(double) * Hq * Wq);
    double *pq = malloc(sizeof(double) * Hq * Wq);
    for (int k = 0; k < n_views; ++k) {
        size_t off = (size_t)k * H * W;
        for (int qy = 0; qy < Hq; ++qy)
            for (int qx = 0; qx < Wq; ++qx) {
                double sum = 0.0;
                int cnt = 0;
                for (int y = 4 * qy; y < 4 * qy + 4 && y < H; ++y)
                    for (int x = 4 * qx; x < 4 * qx + 4 && x < W; ++x) {
                        size_t p = off + (size_t)y * W + x;
                        int dmax = 0;
                        for (int c = 0; c < 3; ++c) {
                            int d = abs((int)rgba_t[4 * p + c] - (int)rgba_prev[4 * p + c]);
                            if (d > dmax) dmax = d;
                        }
                        sum += dmax / 255.0;
                        ++cnt;
                    }
                double m = (sum / cnt) / lambda_t + beta;
                mq[qy * Wq + qx] = m < 1.0 ? m : 1.0;
            }
        for (int qy = 0; qy < Hq; ++qy)
            for (int qx = 0; qx < Wq; ++qx) {
                double best = -1.0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int yy = qy + dy, xx = qx + dx;
                        yy = yy < 0 ? 0 : (yy >= Hq ? Hq - 1 : yy);
                        xx = xx < 0 ? 0 : (xx >= Wq ? Wq - 1 : xx);
                        if (mq[yy * Wq + xx] > best) best = mq[yy * Wq + xx];
                    }
                pq[qy * Wq + qx] = best;
            }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double sx = (x + 0.5) / 4.0 - 0.5, sy = (y + 0.5) / 4.0 - 0.5;
                sx = sx < 0 ? 0 : (sx > Wq - 1 ? Wq - 1 : sx);
                sy = sy < 0 ? 0 : (sy > Hq - 1 ? Hq - 1 : sy);
                int x0 = (int)floor(sx), y0 = (int)floor(sy);
                int x1 = x0 + 1 < Wq ? x0 + 1 : x0, y1 = y0 + 1 < Hq ? y0 + 1 : y0;
                double fx = sx - x0, fy = sy - y0;
                double m = (1 - fy) * ((1 - fx) * pq[y0 * Wq + x0] + fx * pq[y0 * Wq + x1]) +
                           fy * ((1 - fx) * pq[y1 * Wq + x0] + fx * pq[y1 * Wq + x1]);
                size_t p = off + (size_t)y * W + x;
                if (mask_out) mask_out[p] = m;
                float dn = depth_t[p], dp = state_prev[p];
                if (!depth_valid(dp)) state_out[p] = dn;
                else if (!depth_valid(dn)) state_out[p] = dp;
                else state_out[p] = m * (double)dn + (1.0 - m) * (double)dp;
            }
    }
    free(mq);
    free(pq);
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Supplement A.2: the temporal term.                                       */
/* M(p) = max over views of the difference mask at the view's z-buffer       */
/* winner (the splat of every view's mask, channel-wise max); 1 where no     */
/* view covers p (reading: unknown = dynamic).                               */
/* w_tmp(p) = min(beta_t * (w_tmp_prev(p) + w_view_prev(p)) * max(1 - M, 0), */
/*            eta)                                                           */
/* with w_view_prev = sum_k omega_k at the previous frame's crossing.        */
/* The fused depth with the temporal term is orc_fuse_depth with the        */
/* previous output depth and w_tmp as one more input at the same pixel.     */
/* ------------------------------------------------------------------------ */
int orc_temporal_weight(const float *masks, const int32_t *winner, int n_views, int W, int H, int Wt, int Ht,
                        const float *w_tmp_prev, const float *w_view_prev, double beta_t, double eta,
                        double *w_tmp_out, double *mask_out) {
    if (!masks || !winner || n_views <= 0 || !w_tmp_prev || !w_view_prev || !w_tmp_out) return -1;
    size_t np = (size_t)Wt * Ht;
    for (size_t p = 0; p < np; ++p) {
        double M = -1.0;
        for (int k = 0; k < n_views; ++k) {
            int32_t w = winner[(size_t)k * np + p];
            if (w < 0) continue;
            double m = masks[(size_t)k * W * H + (size_t)w];
            if (m > M) M = m;
        }
        if (M < 0.0) M = 1.0;
        if (mask_out) mask_out[p] = M;
        double keep = 1.0 - M;
        keep = keep > 0.0 ? keep : 0.0;
        double w = beta_t * ((double)w_tmp_prev[p] + (double)w_view_prev[p]) * keep;
        w_tmp_out[p] = w < eta ? w : eta;
    }
    return 0;
}

int orc_fuse_depth_temporal(const orc_camera *in_cams, const float *depths, int n_views, const orc_camera *target,
                            int num_samples, double z_near, double z_far, double mu, double weight_const, int window,
                            const float *tmp_depth, const float *tmp_weight, double *out_depth, int32_t *out_index,
                            uint8_t *out_amb, double *out_wview) {
    if (!in_cams || !depths || n_views <= 0 || !target || num_samples < 2 || !(z_near < z_far) || !(mu > 0) ||
        !out_depth || !out_index)
        return -1;
    float (*M)[9] = malloc(sizeof(float[9]) * n_views);
    float (*b)[3] = malloc(sizeof(float[3]) * n_views);
    for (int k = 0; k < n_views; ++k) compose(&in_cams[k], target, M[k], b[k]);
    int64_t n = (int64_t)target->width * target->height;
    fuse_job jb = {in_cams, depths, n_views, target, num_samples, z_near, z_far, mu, weight_const, window,
                   0, NULL, n, out_depth, out_index, out_amb, NULL, M, b, 0, n, tmp_depth, tmp_weight, out_wview};
    fuse_worker(&jb);
    free(M);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1 / Supplement A.3: pixel-sized 3D Gaussians, alpha-composited    */
/* front to back, each input view rendered separately (the rasterisation    */
/* rules of 3D Gaussian splatting, Kerbl et al. 2023, restated).            */
/*                                                                          */
/* Per source pixel (u, v) with valid depth d: an isotropic Gaussian of     */
/* world standard deviation s = scale_px * d / fx_source (its projection    */
/* into the source image spans one pixel), opacity 1, colour = the pixel.   */
/* Its mean projects to (x, y) with depth z = h.z by the splat contract.    */
/* EWA projection into the target (isotropic, so the rotation drops out):   */
/*   Sigma = (scale_px rho)^2 [[1 + a^2, q a b], [q a b, q^2 (1 + b^2)]]     */
/*           + 0.3 I,                                                       */
/*   rho = (fx_t / fx_s) (d / z), a = (x - cx)/fx, b = (y - cy)/fy,          */
/*   q = fy / fx (target intrinsics), 0.3 px^2 the anti-aliasing dilation.   */
/* Radius r = min(ceil(3 sqrt(lambda_max)), max_radius), lambda_max =       */
/* mid + sqrt(max(0.1, mid^2 - det)); covered target pixels                 */
/* i in [ceil(x - r), floor(x + r)], j alike.  Per target pixel the covering */
/* Gaussians are taken in ascending key (bits(z) << 32 | source index):     */
/*   alpha = min(0.99, exp(-0.5 (dx, dy) Sigma^-1 (dx, dy)^T)), (dx, dy) =   */
/*   (x - i, y - j); alpha < 1/255: skipped; T' = T (1 - alpha) < 1e-4:     */
/*   stop before this Gaussian; otherwise C += c alpha T, Z += z alpha T,   */
/*   A += alpha T, T = T'.                                                  */
/* Outputs: colour C (premultiplied, black background), opacity 1 - T,      */
/* depth Z / A (0 where A = 0).                                             */
/* The radius, the covered pixels and the key are integer decisions taken   */
/* in FP32 op for op as the kernel takes them; alpha, colour and depth are  */
/* FP64.  A pixel is flagged ambiguous where some alpha lies within 1e-4    */
/* relative of 1/255, or some T' within 1e-4 relative of 1e-4 (an FP32      */
/* evaluation may decide those thresholds the other way).                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ok;
    float x, y, z, r;
    double cxx, cxy, cyy; /* inverse of Sigma (FP64) */
    double rgb[3];
    uint64_t key;
    int i0, i1, j0, j1;
} gauss_rec;

static gauss_rec gauss_contract(const float A[9], const float c[3], float f_ratio, double f_ratio_d,
                                float scale_px, const float in32[5], const double in64[5], int max_radius,
                                int u, int v, float d, uint32_t rgba, int Wt, int Ht) {
    gauss_rec g;
    memset(&g, 0, sizeof(g));
    if (!depth_valid(d)) return g;
    float m0 = fmaf(A[0], (float)u, fmaf(A[1], (float)v, A[2]));
    float m1 = fmaf(A[3], (float)u, fmaf(A[4], (float)v, A[5]));
    float m2 = fmaf(A[6], (float)u, fmaf(A[7], (float)v, A[8]));
    float h0 = fmaf(d, m0, c[0]);
    float h1 = fmaf(d, m1, c[1]);
    float h2 = fmaf(d, m2, c[2]);
    if (!(h2 > 1e-6f)) return g;
    float x = h0 / h2, y = h1 / h2;
    /* FP32 radius, op for op as the kernel (in32 = fx, fy, cx, cy, fy/fx of the target) */
    float rho = f_ratio * (d / h2);
    float t = scale_px * rho;
    float s2 = t * t;
    float a = (x - in32[2]) / in32[0], b = (y - in32[3]) / in32[1];
    float q = in32[4];
    float aa = a * a, bb = b * b, ab = a * b, qq = q * q;
    float sxx = s2 * (1.0f + aa) + 0.3f;
    float sxy = s2 * (q * ab);
    float syy = s2 * (qq * (1.0f + bb)) + 0.3f;
    float p1 = sxx * syy, p2 = sxy * sxy;
    float det = p1 - p2;
    if (!(det > 0.0f)) return g;
    float mid = 0.5f * (sxx + syy);
    float disc = mid * mid - det;
    disc = disc > 0.1f ? disc : 0.1f;
    float lam = mid + sqrtf(disc);
    float rr = ceilf(3.0f * sqrtf(lam));
    if (!(rr <= (float)max_radius)) rr = (float)max_radius;
    float lo_x = ceilf(x - rr), hi_x = floorf(x + rr);
    float lo_y = ceilf(y - rr), hi_y = floorf(y + rr);
    if (lo_x < 0.0f) lo_x = 0.0f;
    if (lo_y < 0.0f) lo_y = 0.0f;
    if (hi_x > (float)(Wt - 1)) hi_x = (float)(Wt - 1);
    if (hi_y > (float)(Ht - 1)) hi_y = (float)(Ht - 1);
    if (!(lo_x <= hi_x) || !(lo_y <= hi_y)) return g;
    /* FP64 covariance and its inverse (in64 = fx, fy, cx, cy, fy/fx) */
    double rho_d = f_ratio_d * ((double)d / (double)h2);
    double s2d = ((double)scale_px * rho_d) * ((double)scale_px * rho_d);
    double ad = ((double)x - in64[2]) / in64[0], bd = ((double)y - in64[3]) / in64[1], qd = in64[4];
    double Sxx = s2d * (1.0 + ad * ad) + 0.3;
    double Sxy = s2d * qd * ad * bd;
    double Syy = s2d * qd * qd * (1.0 + bd * bd) + 0.3;
    double detd = Sxx * Syy - Sxy * Sxy;
    g.cxx = Syy / detd;
    g.cxy = -Sxy / detd;
    g.cyy = Sxx / detd;
    g.ok = 1;
    g.x = x; g.y = y; g.z = h2; g.r = rr;
    g.i0 = (int)lo_x; g.i1 = (int)hi_x; g.j0 = (int)lo_y; g.j1 = (int)hi_y;
    for (int ch = 0; ch < 3; ++ch) g.rgb[ch] = (double)((rgba >> (8 * ch)) & 0xffu) / 255.0;
    return g;
}

typedef struct {
    uint64_t key;
    int32_t rec;
} gauss_ref;

static int cmp_gauss_ref(const void *pa, const void *pb) {
    uint64_t a = ((const gauss_ref *)pa)->key, b = ((const gauss_ref *)pb)->key;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* pixels: target pixel indices (j * Wt + i) to evaluate, or NULL for all (n_pixels ignored).
 * Outputs [n_views][P]: color [.][.][4] (r, g, b premultiplied, opacity), depth, amb. */
int orc_gauss_splat(const orc_camera *in_cams, const float *depths, const uint32_t *rgba, int n_views,
                    const orc_camera *target, float scale_px, int max_radius, const int32_t *pixels,
                    int64_t n_pixels, double *color, double *depth_out, uint8_t *amb) {
    if (!in_cams || !depths || !rgba || n_views <= 0 || !target || !color || !depth_out) return -1;
    if (!(scale_px > 0.0f) || max_radius < 1) return -1;
    const int Wt = target->width, Ht = target->height;
    const int64_t np = (int64_t)Wt * Ht;
    const int64_t P = pixels ? n_pixels : np;
    /* slot of each target pixel among the evaluated ones (-1: not evaluated) */
    int64_t *slot = malloc(sizeof(int64_t) * (size_t)np);
    for (int64_t p = 0; p < np; ++p) slot[p] = pixels ? -1 : p;
    if (pixels)
        for (int64_t s = 0; s < P; ++s) slot[pixels[s]] = s;
    const float in32[5] = {(float)target->fx, (float)target->fy, (float)target->cx, (float)target->cy,
                           (float)(target->fy / target->fx)};
    const double in64[5] = {target->fx, target->fy, target->cx, target->cy, target->fy / target->fx};
    size_t in_off = 0;
    for (int k = 0; k < n_views; ++k) {
        const orc_camera *vc = &in_cams[k];
        const int W = vc->width, H = vc->height;
        float Am[9], cm[3];
        compose(target, vc, Am, cm);
        const float f_ratio = (float)(target->fx / vc->fx);
        const double f_ratio_d = target->fx / vc->fx;
        gauss_rec *rec = malloc(sizeof(gauss_rec) * (size_t)W * H);
        int64_t *count = calloc((size_t)P + 1, sizeof(int64_t));
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                size_t s = (size_t)v * W + u;
                rec[s] = gauss_contract(Am, cm, f_ratio, f_ratio_d, scale_px, in32, in64, max_radius, u, v,
                                        depths[in_off + s], rgba[in_off + s], Wt, Ht);
                rec[s].key = make_key(rec[s].z, (uint32_t)s);
                if (!rec[s].ok) continue;
                for (int j = rec[s].j0; j <= rec[s].j1; ++j)
                    for (int i = rec[s].i0; i <= rec[s].i1; ++i) {
                        int64_t sl = slot[(int64_t)j * Wt + i];
                        if (sl >= 0) ++count[sl + 1];
                    }
            }
        for (int64_t s = 0; s < P; ++s) count[s + 1] += count[s];
        gauss_ref *list = malloc(sizeof(gauss_ref) * (size_t)(count[P] > 0 ? count[P] : 1));
        int64_t *fill = malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
        for (int64_t s = 0; s < P; ++s) fill[s] = count[s];
        for (size_t s = 0; s < (size_t)W * H; ++s) {
            if (!rec[s].ok) continue;
            for (int j = rec[s].j0; j <= rec[s].j1; ++j)
                for (int i = rec[s].i0; i <= rec[s].i1; ++i) {
                    int64_t sl = slot[(int64_t)j * Wt + i];
                    if (sl >= 0) {
                        list[fill[sl]].key = rec[s].key;
                        list[fill[sl]].rec = (int32_t)s;
                        ++fill[sl];
                    }
                }
        }
        for (int64_t s = 0; s < P; ++s) {
            const int64_t p = pixels ? pixels[s] : s;
            const double pi = (double)(p % Wt), pj = (double)(p / Wt);
            gauss_ref *L = list + count[s];
            const int64_t n = count[s + 1] - count[s];
            qsort(L, (size_t)n, sizeof(gauss_ref), cmp_gauss_ref);
            double T = 1.0, C[3] = {0.0, 0.0, 0.0}, Z = 0.0, Acc = 0.0;
            int am = 0;
            for (int64_t e = 0; e < n; ++e) {
                const gauss_rec *g = &rec[L[e].rec];
                double dx = (double)g->x - pi, dy = (double)g->y - pj;
                double power = -0.5 * (g->cxx * dx * dx + g->cyy * dy * dy) - g->cxy * dx * dy;
                if (power > 0.0) continue;
                double al = exp(power);
                al = al < 0.99 ? al : 0.99;
                if (fabs(al - 1.0 / 255.0) <= 1e-4 / 255.0) am = 1;
                if (al < 1.0 / 255.0) continue;
                double Tn = T * (1.0 - al);
                if (fabs(Tn - 1e-4) <= 1e-8) am = 1;
                if (Tn < 1e-4) break;
                for (int ch = 0; ch < 3; ++ch) C[ch] += g->rgb[ch] * al * T;
                Z += (double)g->z * al * T;
                Acc += al * T;
                T = Tn;
            }
            double *o = color + ((size_t)k * P + s) * 4;
            o[0] = C[0]; o[1] = C[1]; o[2] = C[2]; o[3] = 1.0 - T;
            depth_out[(size_t)k * P + s] = Acc > 0.0 ? Z / Acc : 0.0;
            if (amb) amb[(size_t)k * P + s] = (uint8_t)am;
        }
        free(rec);
        free(count);
        free(list);
        free(fill);
        in_off += (size_t)W * H;
    }
    free(slot);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 and the supplement's network-input list: the (9K + 1) x H x W   */
/* input of the blending network, and the blend of Eqs. 4-5 with L_Depth.   */
/*                                                                          */
/* Channels, in the listed order: forward-rendered colours (3K, k-major,    */
/* RGB / 255), their depths D_k (K), alphas (K), the TSDF depth D (1), then */
/* per view k: n . d_k (K), r_t . d_k (K), |c_k - c_t| (K), z_k . z_t (K).  */
/* With P the target-camera point of pixel p at depth D(p), n the normal of */
/* D at p, d_k the unit ray from view k's centre to P, r_t = P / |P|, z the */
/* cameras' optical axes; all vectors in the target camera frame.          */
/* n = (P(i+1,j) - P(i-1,j)) x (P(i,j+1) - P(i,j-1)), turned to face the     */
/* camera and normalised; 0 where p or one of its four neighbours has no    */
/* depth (or lies outside the image).  The differences are formed as        */
/*   dx: (delta (i - cx) + sigma) / fx, delta (j - cy) / fy, delta          */
/* with delta = D+ - D-, sigma = D+ + D- (the same vector, written without  */
/* subtracting two large coordinates).  n . d_k and r_t . d_k are 0 where   */
/* D(p) is 0.                                                               */
/* ------------------------------------------------------------------------ */
static void target_point(const orc_camera *t, double i, double j, double D, double P[3]) {
    P[0] = D * (i - t->cx) / t->fx;
    P[1] = D * (j - t->cy) / t->fy;
    P[2] = D;
}

static void centre_in_target(const orc_camera *t, const orc_camera *c, double o[3]) {
    double w[3];
    for (int r = 0; r < 3; ++r) w[r] = -(c->R[0 + r] * c->t[0] + c->R[3 + r] * c->t[1] + c->R[6 + r] * c->t[2]);
    for (int r = 0; r < 3; ++r) o[r] = t->R[3 * r + 0] * w[0] + t->R[3 * r + 1] * w[1] + t->R[3 * r + 2] * w[2] + t->t[r];
}

int orc_blend_features(const orc_camera *in_cams, int n_views, const orc_camera *target,
                       const uint32_t *warped_rgba, const float *warped_depth, const uint8_t *alpha,
                       const float *fused, double *features) {
    if (!in_cams || n_views <= 0 || !target || !warped_rgba || !warped_depth || !alpha || !fused || !features)
        return -1;
    const int K = n_views, W = target->width, H = target->height;
    const size_t np = (size_t)W * H;
    double (*ck)[3] = malloc(sizeof(double[3]) * K);
    double *dist = malloc(sizeof(double) * K), *axis = malloc(sizeof(double) * K);
    double ct_world[3];
    for (int r = 0; r < 3; ++r)
        ct_world[r] = -(target->R[0 + r] * target->t[0] + target->R[3 + r] * target->t[1] + target->R[6 + r] * target->t[2]);
    for (int k = 0; k < K; ++k) {
        centre_in_target(target, &in_cams[k], ck[k]);
        double cw[3], s = 0.0, a = 0.0;
        for (int r = 0; r < 3; ++r)
            cw[r] = -(in_cams[k].R[0 + r] * in_cams[k].t[0] + in_cams[k].R[3 + r] * in_cams[k].t[1] +
                      in_cams[k].R[6 + r] * in_cams[k].t[2]);
        for (int r = 0; r < 3; ++r) {
            s += (cw[r] - ct_world[r]) * (cw[r] - ct_world[r]);
            a += in_cams[k].R[6 + r] * target->R[6 + r];
        }
        dist[k] = sqrt(s);
        axis[k] = a;
    }
#define FEAT(c, p) features[(size_t)(c) * np + (p)]
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            const size_t p = (size_t)j * W + i;
            for (int k = 0; k < K; ++k) {
                const size_t o = (size_t)k * np + p;
                const uint32_t c = warped_rgba[o];
                for (int ch = 0; ch < 3; ++ch) FEAT(3 * k + ch, p) = (double)((c >> (8 * ch)) & 0xffu) / 255.0;
                FEAT(3 * K + k, p) = (double)warped_depth[o];
                FEAT(4 * K + k, p) = (double)alpha[o];
                FEAT(5 * K + 1 + 2 * K + k, p) = dist[k];
                FEAT(5 * K + 1 + 3 * K + k, p) = axis[k];
            }
            const double D = (double)fused[p];
            FEAT(5 * K, p) = D;
            const int have = depth_valid(fused[p]);
            double n[3] = {0.0, 0.0, 0.0};
            if (have && i > 0 && i < W - 1 && j > 0 && j < H - 1 && depth_valid(fused[p - 1]) &&
                depth_valid(fused[p + 1]) && depth_valid(fused[p - W]) && depth_valid(fused[p + W])) {
                const double dh = (double)fused[p + 1] - (double)fused[p - 1];
                const double sh = (double)fused[p + 1] + (double)fused[p - 1];
                const double dv = (double)fused[p + W] - (double)fused[p - W];
                const double sv = (double)fused[p + W] + (double)fused[p - W];
                const double a[3] = {(dh * (i - target->cx) + sh) / target->fx, dh * (j - target->cy) / target->fy, dh};
                const double b[3] = {dv * (i - target->cx) / target->fx, (dv * (j - target->cy) + sv) / target->fy, dv};
                n[0] = a[1] * b[2] - a[2] * b[1];
                n[1] = a[2] * b[0] - a[0] * b[2];
                n[2] = a[0] * b[1] - a[1] * b[0];
                double P[3];
                target_point(target, i, j, D, P);
                if (n[0] * P[0] + n[1] * P[1] + n[2] * P[2] > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
                const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                if (len > 0.0) { n[0] /= len; n[1] /= len; n[2] /= len; }
            }
            for (int k = 0; k < K; ++k) {
                double nd = 0.0, rd = 0.0;
                if (have) {
                    double P[3], d[3];
                    target_point(target, i, j, D, P);
                    for (int r = 0; r < 3; ++r) d[r] = P[r] - ck[k][r];
                    const double ld = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    const double lp = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
                    for (int r = 0; r < 3; ++r) {
                        nd += n[r] * d[r] / ld;
                        rd += P[r] / lp * d[r] / ld;
                    }
                }
                FEAT(5 * K + 1 + k, p) = nd;
                FEAT(5 * K + 1 + K + k, p) = rd;
            }
        }
#undef FEAT
    free(ck);
    free(dist);
    free(axis);
    return 0;
}

/* Eq. 4 (denominator read as the sum over views), Eq. 5 and L_Depth:       */
/*   I_FG = sum_k I_k a_k w_k / sum_k a_k w_k   (0 where the sum is 0)       */
/*   I    = (1 - w_BG) I_FG + w_BG I_BG                                      */
/*   L_Depth = 1/(H W K) sum_p | D(p) - sum_k D_k a_k w_k / sum_k a_k w_k |  */
/* w [K][H][W], w_bg [H][W], i_bg [3][H][W]; out [3][H][W].                  */
int orc_blend(int n_views, int W, int H, const uint32_t *warped_rgba, const uint8_t *alpha,
              const float *warped_depth, const float *fused, const double *w, const double *w_bg,
              const double *i_bg, double *out, double *l_depth) {
    if (n_views <= 0 || W <= 0 || H <= 0 || !warped_rgba || !alpha || !warped_depth || !fused || !w || !w_bg ||
        !i_bg || !out)
        return -1;
    const size_t np = (size_t)W * H;
    double L = 0.0;
    for (size_t p = 0; p < np; ++p) {
        double den = 0.0, num[3] = {0.0, 0.0, 0.0}, dnum = 0.0;
        for (int k = 0; k < n_views; ++k) {
            const size_t o = (size_t)k * np + p;
            const double aw = (double)alpha[o] * w[o];
            const uint32_t c = warped_rgba[o];
            for (int ch = 0; ch < 3; ++ch) num[ch] += (double)((c >> (8 * ch)) & 0xffu) / 255.0 * aw;
            dnum += (double)warped_depth[o] * aw;
            den += aw;
        }
        for (int ch = 0; ch < 3; ++ch) {
            const double fg = den > 0.0 ? num[ch] / den : 0.0;
            out[(size_t)ch * np + p] = (1.0 - w_bg[p]) * fg + w_bg[p] * i_bg[(size_t)ch * np + p];
        }
        L += fabs((double)fused[p] - (den > 0.0 ? dnum / den : 0.0));
    }
    if (l_depth) *l_depth = L / ((double)np * n_views);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Supplement A.1, the paper's own raymarch: advance along the ray by 0.8 s */
/* until s changes sign, then three bisection steps.                        */
/*                                                                          */
/* Every quantity on the path decides where the next sample lands, so the   */
/* whole march is taken in FP32, each operation rounded as written, the     */
/* kernel's precision (no FP64 step: an FP64 trajectory would drift from    */
/* any FP32 one and visit other pixels).  Readings:                         */
/*   s_n = S / W (the weighted mean of clamp(sdf, -1, 1), sdf = (d - z)/mu);  */
/*   the step is 0.8 mu max(s_n, min_frac) where W > 0 (min_frac > 0 keeps   */
/*   the march moving: with s_n = (d - z)/mu the plain 0.8 s step would     */
/*   approach the surface geometrically and never cross it) and 0.8 mu     */
/*   (a full truncation) where no view sees the point (W = 0);             */
/*   a crossing is a sample with W > 0 and S <= 0 after one with W > 0 and   */
/*   S > 0; bisection keeps the lower half where W > 0 and S > 0 at the      */
/*   midpoint, else the upper; the depth is the final bracket's midpoint.   */
/*   The march starts at z_near, stops past z_far or after max_steps         */
/*   samples (no crossing: depth 0).                                        */
/* The weights are the confidence weights of Supplement A.1 in FP32:        */
/*   nu = fma(t, t, nu) over the window in raster order, t = min(|dc - dn|,  */
/*   mu) (mu for an invalid neighbour), omega = min(wconst / sqrt(nu / w^2), */
/*   1) (1 where nu = 0, 0 for an invalid centre).                          */
/* ------------------------------------------------------------------------ */
float orc_weight_f32(const float *depth, int H, int W, int u, int v, float mu, float wconst, int window,
                     float inv_w2) {
    float dc = depth[(size_t)v * W + u];
    if (!depth_valid(dc)) return 0.0f;
    int r = window / 2;
    float nu = 0.0f;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            int q = v + dy, p = u + dx;
            q = q < 0 ? 0 : (q >= H ? H - 1 : q);
            p = p < 0 ? 0 : (p >= W ? W - 1 : p);
            float dn = depth[(size_t)q * W + p];
            float t = depth_valid(dn) ? fminf(fabsf(dc - dn), mu) : mu;
            nu = fmaf(t, t, nu);
        }
    if (!(nu > 0.0f)) return 1.0f;
    float w = wconst / sqrtf(nu * inv_w2);
    return w < 1.0f ? w : 1.0f;
}

typedef struct {
    const orc_camera *in_cams; const float *depths; int K;
    const orc_camera *target;
    float zn, zf, inv_mu, c08mu, min_frac, mu, wconst, inv_w2; int window, max_steps;
    float (*M)[9]; float (*b)[3];
    float *wmap; /* [K][H][W] FP32 weights */
} sphere_job;

static void sphere_eval(const sphere_job *jb, const float (*a)[3], float z, float *S_out, float *W_out) {
    float S = 0.0f, Wt = 0.0f;
    for (int k = 0; k < jb->K; ++k) {
        const orc_camera *vc = &jb->in_cams[k];
        float h2 = fmaf(z, a[k][2], jb->b[k][2]);
        if (!(h2 > 1e-6f)) continue;
        float h0 = fmaf(z, a[k][0], jb->b[k][0]);
        float h1 = fmaf(z, a[k][1], jb->b[k][1]);
        double u = nearest_of_quotient(h0, h2), v = nearest_of_quotient(h1, h2);
        if (u < 0 || v < 0 || u > vc->width - 1 || v > vc->height - 1) continue;
        size_t o = (size_t)k * vc->width * vc->height + (size_t)v * vc->width + (size_t)u;
        float d = jb->depths[o];
        if (!depth_valid(d)) continue;   /* stored as (0, 0): sdf < -1 */
        float sdf = (d - h2) * jb->inv_mu;
        if (!(sdf >= -1.0f)) continue;
        float w = jb->wmap[o];
        S = fmaf(w, sdf < 1.0f ? sdf : 1.0f, S);
        Wt = Wt + w;
    }
    *S_out = S;
    *W_out = Wt;
}

int orc_fuse_depth_sphere(const orc_camera *in_cams, const float *depths, int n_views, const orc_camera *target,
                          double z_near, double z_far, double mu, double weight_const, int window, int max_steps,
                          double min_frac, float *out_depth, int32_t *out_evals) {
    if (!in_cams || !depths || n_views <= 0 || !target || !(z_near < z_far) || !(mu > 0) || window < 1 ||
        !(window & 1) || max_steps < 1 || !(min_frac > 0) || !out_depth)
        return -1;
    sphere_job jb;
    jb.in_cams = in_cams; jb.depths = depths; jb.K = n_views; jb.target = target;
    /* the parameters as FP32 values first (the kernel receives them so), constants derived in FP64 */
    const float mu32 = (float)mu;
    jb.zn = (float)z_near; jb.zf = (float)z_far; jb.inv_mu = (float)(1.0 / (double)mu32);
    jb.c08mu = (float)(0.8 * (double)mu32);
    jb.min_frac = (float)min_frac; jb.mu = mu32; jb.wconst = (float)weight_const;
    jb.inv_w2 = (float)(1.0 / ((double)window * (double)window));
    jb.window = window; jb.max_steps = max_steps;
    jb.M = malloc(sizeof(float[9]) * n_views);
    jb.b = malloc(sizeof(float[3]) * n_views);
    for (int k = 0; k < n_views; ++k) compose(&in_cams[k], target, jb.M[k], jb.b[k]);
    size_t off = 0;
    for (int k = 0; k < n_views; ++k) off += (size_t)in_cams[k].width * in_cams[k].height;
    jb.wmap = malloc(sizeof(float) * (off > 0 ? off : 1));
    off = 0;
    for (int k = 0; k < n_views; ++k) {
        const int W = in_cams[k].width, H = in_cams[k].height;
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u)
                jb.wmap[off + (size_t)v * W + u] =
                    orc_weight_f32(depths + off, H, W, u, v, jb.mu, jb.wconst, window, jb.inv_w2);
        off += (size_t)W * H;
    }
    float (*a)[3] = malloc(sizeof(float[3]) * n_views);
    for (int j = 0; j < target->height; ++j)
        for (int i = 0; i < target->width; ++i) {
            for (int k = 0; k < n_views; ++k) {
                const float *M = jb.M[k];
                a[k][0] = fmaf(M[0], (float)i, fmaf(M[1], (float)j, M[2]));
                a[k][1] = fmaf(M[3], (float)i, fmaf(M[4], (float)j, M[5]));
                a[k][2] = fmaf(M[6], (float)i, fmaf(M[7], (float)j, M[8]));
            }
            float z = jb.zn, z_prev = 0.0f, S_prev = 0.0f, W_prev = 0.0f, out = 0.0f;
            int have_prev = 0, evals = 0;
            for (int it = 0; it < max_steps && z <= jb.zf; ++it) {
                float S, Wt;
                sphere_eval(&jb, (const float (*)[3])a, z, &S, &Wt);
                ++evals;
                if (have_prev && W_prev > 0.0f && Wt > 0.0f && S_prev > 0.0f && S <= 0.0f) {
                    float lo = z_prev, hi = z;
                    for (int bstep = 0; bstep < 3; ++bstep) {
                        float m = 0.5f * (lo + hi), Sm, Wm;
                        sphere_eval(&jb, (const float (*)[3])a, m, &Sm, &Wm);
                        ++evals;
                        if (Wm > 0.0f && Sm > 0.0f) lo = m;
                        else hi = m;
                    }
                    out = 0.5f * (lo + hi);
                    break;
                }
                float stepn = 1.0f;
                if (Wt > 0.0f) {
                    float sn = S / Wt;
                    stepn = sn > jb.min_frac ? sn : jb.min_frac;
                }
                S_prev = S; W_prev = Wt; z_prev = z; have_prev = 1;
                z = z + jb.c08mu * stepn;
            }
            out_depth[(size_t)j * target->width + i] = out;
            if (out_evals) out_evals[(size_t)j * target->width + i] = evals;
        }
    free(a);
    free(jb.M);
    free(jb.b);
    free(jb.wmap);
    return 0;
}
