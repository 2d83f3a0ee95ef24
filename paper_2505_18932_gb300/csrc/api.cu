// Host side of the C ABI declared in include/gvs.h: argument checks, FP64
// composition of the per-view FP32 contract coefficients, kernel dispatch.
// Built with -ffp-contract=off so that the FP64 composition is evaluated in
// exactly the documented order.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "blend_internal.cuh"
#include "bounds_check.cuh"
#include "sphere_internal.cuh"
#include "gauss_internal.cuh"
#include "gvs_internal.cuh"

namespace {

thread_local char g_err[512] = "";

// NVTX range around each entry point (a no-op unless a profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

gvs_status fail(gvs_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

gvs_status cuda_fail(cudaError_t e, const char *where) {
    return fail(GVS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

bool camera_ok(const gvs_camera *c) {
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > GVS_MAX_DIM || c->height > GVS_MAX_DIM) return false;
    if (!(isfinite(c->fx) && isfinite(c->fy) && isfinite(c->cx) && isfinite(c->cy))) return false;
    if (!(c->fx > 0.0) || !(c->fy > 0.0)) return false;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(c->R[i])) return false;
    for (int i = 0; i < 3; ++i)
        if (!isfinite(c->t[i])) return false;
    return true;
}

// FP64 composition in the order documented in gvs.h, rounded once to FP32.
gvs::ViewXform compose(const gvs_camera &to, const gvs_camera &from) {
    double Q[9], g[3], N[9], bb[3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Q[3 * r + c] = to.R[3 * r + 0] * from.R[3 * c + 0] + to.R[3 * r + 1] * from.R[3 * c + 1] +
                           to.R[3 * r + 2] * from.R[3 * c + 2];
    for (int r = 0; r < 3; ++r)
        g[r] = to.t[r] - (Q[3 * r + 0] * from.t[0] + Q[3 * r + 1] * from.t[1] + Q[3 * r + 2] * from.t[2]);
    for (int c = 0; c < 3; ++c) {
        N[0 + c] = to.fx * Q[0 + c] + to.cx * Q[6 + c];
        N[3 + c] = to.fy * Q[3 + c] + to.cy * Q[6 + c];
        N[6 + c] = Q[6 + c];
    }
    bb[0] = to.fx * g[0] + to.cx * g[2];
    bb[1] = to.fy * g[1] + to.cy * g[2];
    bb[2] = g[2];
    gvs::ViewXform x;
    for (int r = 0; r < 3; ++r) {
        x.M[3 * r + 0] = (float)(N[3 * r + 0] / from.fx);
        x.M[3 * r + 1] = (float)(N[3 * r + 1] / from.fy);
        x.M[3 * r + 2] = (float)((N[3 * r + 2] - (N[3 * r + 0] * from.cx) / from.fx) - (N[3 * r + 1] * from.cy) / from.fy);
        x.b[r] = (float)bb[r];
    }
    return x;
}

size_t align_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

bool views_ok(const gvs_camera *cams, int32_t n, int32_t *W, int32_t *H) {
    if (n < 0 || n > GVS_MAX_VIEWS) return false;
    if (n == 0) { *W = *H = 0; return true; }
    if (!cams) return false;
    for (int k = 0; k < n; ++k) {
        if (!camera_ok(&cams[k])) return false;
        if (cams[k].width != cams[0].width || cams[k].height != cams[0].height) return false;
    }
    *W = cams[0].width;
    *H = cams[0].height;
    return true;
}

}  // namespace

namespace gvs {

int device_sm_count() {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        cache[dev] = sms;
    }
    return cache[dev];
}

}  // namespace gvs

extern "C" {

const char *gvs_version(void) { return "gvs 0.1.0 (sm_103a)"; }

const char *gvs_status_string(gvs_status s) {
    switch (s) {
        case GVS_OK: return "ok";
        case GVS_ERR_INVALID_ARG: return "invalid argument";
        case GVS_ERR_UNSUPPORTED: return "unsupported";
        case GVS_ERR_WORKSPACE: return "workspace too small or misaligned";
        case GVS_ERR_CUDA: return "CUDA error";
        case GVS_ERR_DEVICE: return "no usable CUDA device";
    }
    return "unknown status";
}

const char *gvs_last_error(void) { return g_err; }

gvs_status gvs_refine_depth(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t,
                            void *depth_state, uint8_t *mask, int32_t n_views, int32_t width, int32_t height,
                            const gvs_refine_params *params, void *stream) {
    const Range nvtx_range("gvs_refine_depth");
    if (!params) return fail(GVS_ERR_INVALID_ARG, "refine: params is NULL");
    if (n_views < 0 || n_views > GVS_MAX_VIEWS) return fail(GVS_ERR_INVALID_ARG, "refine: n_views out of range");
    if (width < 1 || height < 1 || width > GVS_MAX_DIM || height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "refine: image size out of range");
    if (!(params->tau >= 0.0f && params->tau <= 1.0f)) return fail(GVS_ERR_INVALID_ARG, "refine: tau not in [0,1]");
    if (params->depth_dtype != GVS_F32 && params->depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "refine: depth_dtype must be GVS_F32 or GVS_F16");
    if (n_views == 0) return GVS_OK;
    if (!rgba_t || !depth_t || !depth_state) return fail(GVS_ERR_INVALID_ARG, "refine: NULL array");
    if (!aligned(rgba_t, 16) || !aligned(depth_t, 16) || !aligned(depth_state, 16) ||
        (rgba_prev && !aligned(rgba_prev, 16)) || (mask && !aligned(mask, 16)))
        return fail(GVS_ERR_INVALID_ARG, "refine: arrays must be 16-byte aligned");
    const int threshold = (int)floor(255.0 * (double)params->tau);
    const int64_t n = (int64_t)n_views * width * height;
    cudaError_t e = gvs::launch_refine(rgba_t, rgba_prev, depth_t, depth_state, mask, n, threshold,
                                       params->depth_dtype, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "refine launch");
    return GVS_OK;
}

size_t gvs_refine_soft_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
    if (n_views < 0 || width < 0 || height < 0) return 0;
    return align_up(2 * (size_t)n_views * (size_t)((width + 3) / 4) * (size_t)((height + 3) / 4) * sizeof(float), 256);
}

gvs_status gvs_refine_depth_soft(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t,
                                 void *depth_state, float *mask, int32_t n_views, int32_t width, int32_t height,
                                 const gvs_refine_soft_params *params, void *workspace, size_t workspace_bytes,
                                 void *stream) {
    const Range nvtx_range("gvs_refine_depth_soft");
    if (!params) return fail(GVS_ERR_INVALID_ARG, "soft refine: params is NULL");
    if (n_views < 0 || n_views > GVS_MAX_VIEWS) return fail(GVS_ERR_INVALID_ARG, "soft refine: n_views out of range");
    if (width < 1 || height < 1 || width > GVS_MAX_DIM || height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "soft refine: image size out of range");
    if (!(isfinite(params->beta) && params->beta >= 0.0f && params->beta <= 1.0f))
        return fail(GVS_ERR_INVALID_ARG, "soft refine: beta must be in [0, 1]");
    if (!(isfinite(params->lambda_t) && params->lambda_t > 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "soft refine: lambda_t must be > 0");
    if (params->depth_dtype != GVS_F32 && params->depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "soft refine: depth_dtype must be GVS_F32 or GVS_F16");
    if (n_views == 0) return GVS_OK;
    if (!rgba_t || !rgba_prev || !depth_t || !depth_state)
        return fail(GVS_ERR_INVALID_ARG, "soft refine: rgba_t, rgba_prev, depth_t and depth_state are required");
    const void *arrs[] = {rgba_t, rgba_prev, depth_t, depth_state, mask};
    for (const void *q : arrs)
        if (q && !aligned(q, 16)) return fail(GVS_ERR_INVALID_ARG, "soft refine: arrays must be 16-byte aligned");
    const size_t need = gvs_refine_soft_workspace_bytes(n_views, width, height);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "soft refine: workspace needs %zu bytes, 256-byte aligned", need);
    cudaError_t e = gvs::launch_refine_soft(rgba_t, rgba_prev, depth_t, depth_state, mask, n_views, width, height,
                                            params->beta, params->lambda_t, params->depth_dtype,
                                            reinterpret_cast<float *>(workspace), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "soft refine: launch");
    return GVS_OK;
}

gvs_status gvs_select_views(const gvs_camera *cams, int32_t n, const gvs_camera *target, int32_t k,
                            int32_t *out_idx) {
    const Range nvtx_range("gvs_select_views");
    if (!cams || !target || !out_idx || n < 1 || k < 1 || k > n)
        return fail(GVS_ERR_INVALID_ARG, "select views: need cameras, a target, out_idx and 1 <= k <= n");
    for (int i = 0; i < n; ++i)
        if (!camera_ok(&cams[i])) return fail(GVS_ERR_INVALID_ARG, "select views: camera %d invalid", i);
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "select views: target camera invalid");
    auto centre = [](const gvs_camera &c, double C[3]) {  // C = -R^T t
        for (int a = 0; a < 3; ++a) C[a] = -(c.R[0 * 3 + a] * c.t[0] + c.R[1 * 3 + a] * c.t[1] + c.R[2 * 3 + a] * c.t[2]);
    };
    double Ct[3];
    centre(*target, Ct);
    std::vector<std::pair<double, int>> d((size_t)n);
    for (int i = 0; i < n; ++i) {
        double C[3];
        centre(cams[i], C);
        const double dx = C[0] - Ct[0], dy = C[1] - Ct[1], dz = C[2] - Ct[2];
        d[(size_t)i] = {dx * dx + dy * dy + dz * dz, i};
    }
    std::stable_sort(d.begin(), d.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first < b.first;
    });
    for (int i = 0; i < k; ++i) out_idx[i] = d[(size_t)i].second;
    return GVS_OK;
}

size_t gvs_fuse_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
    if (n_views < 0 || width < 0 || height < 0) return 0;
    return gvs::map_layout(n_views, width, height).total;
}

}  // extern "C"

namespace {

gvs_status check_fuse_common(const gvs_camera *in_cams, int32_t n_views, const gvs_camera *target,
                             const gvs_fuse_params *params, const float *fused_depth, const int16_t *crossing,
                             int32_t *W, int32_t *H) {
    if (!params) return fail(GVS_ERR_INVALID_ARG, "fuse: params is NULL");
    if (!views_ok(in_cams, n_views, W, H))
        return fail(GVS_ERR_INVALID_ARG, "fuse: input cameras invalid, of different sizes, or n_views out of range");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "fuse: target camera invalid");
    const gvs_fuse_params &p = *params;
    if (p.num_samples < 2 || p.num_samples > GVS_MAX_SAMPLES) return fail(GVS_ERR_INVALID_ARG, "fuse: num_samples");
    if (!(isfinite(p.z_near) && isfinite(p.z_far) && p.z_near > 0.0f && p.z_near < p.z_far))
        return fail(GVS_ERR_INVALID_ARG, "fuse: need 0 < z_near < z_far");
    if (!(isfinite(p.mu) && p.mu > 0.0f)) return fail(GVS_ERR_INVALID_ARG, "fuse: mu must be > 0");
    if (p.normalize != 0 && p.normalize != 1) return fail(GVS_ERR_INVALID_ARG, "fuse: normalize must be 0 or 1");
    if (p.depth_dtype != GVS_F32 && p.depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "fuse: depth_dtype must be GVS_F32 or GVS_F16");
    if (p.map_dtype != GVS_F32 && p.map_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "fuse: map_dtype must be GVS_F32 or GVS_F16");
    if (p.variant < 0 || p.variant > 6) return fail(GVS_ERR_INVALID_ARG, "fuse: variant must be in [0, 6]");
    if (!fused_depth) return fail(GVS_ERR_INVALID_ARG, "fuse: fused_depth is NULL");
    if (!aligned(fused_depth, 16) || (crossing && !aligned(crossing, 16)))
        return fail(GVS_ERR_INVALID_ARG, "fuse: arrays must be 16-byte aligned");
    return GVS_OK;
}

gvs_status check_weight_params(float mu, float weight_const, int32_t window) {
    if (!(isfinite(mu) && mu > 0.0f)) return fail(GVS_ERR_INVALID_ARG, "weight map: mu must be > 0");
    if (!(isfinite(weight_const) && weight_const > 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "weight map: weight_const must be > 0");
    if (window < 1 || window > GVS_MAX_WINDOW || (window & 1) == 0)
        return fail(GVS_ERR_INVALID_ARG, "weight map: window must be odd in [1, %d]", GVS_MAX_WINDOW);
    return GVS_OK;
}

gvs::FuseArgs fuse_args(const gvs_camera *in_cams, const void *map, int32_t n_views, int32_t W, int32_t H,
                        const gvs_camera *target, const gvs_fuse_params &p, float *fused, int16_t *crossing) {
    gvs::FuseArgs a;
    memset(&a, 0, sizeof(a));
    const gvs::MapLayout L = gvs::map_layout(n_views, W, H);
    const char *m = reinterpret_cast<const char *>(map);
    if (n_views > 0) {
        a.dw = m + L.off_dw;
        for (int l = 0; l < gvs::kBoundLevels; ++l) a.ob[l] = reinterpret_cast<const gvs::DepthBound *>(m + L.off_O[l]);
        a.tg = reinterpret_cast<const gvs::DepthBound *>(m + L.off_g);
    }
    for (int l = 0; l < gvs::kBoundLevels; ++l) {
        a.tw[l] = L.tw[l];
        a.th[l] = L.th[l];
    }
    a.K = n_views;
    a.W = W;
    a.H = H;
    a.Wt = target->width;
    a.Ht = target->height;
    a.D = p.num_samples;
    a.zn = p.z_near;
    a.dz = (float)(((double)p.z_far - (double)p.z_near) / (double)(p.num_samples - 1));
    a.inv_mu = (float)(1.0 / (double)p.mu);
    a.behind = (float)(1.0001 * (double)p.mu);
    a.normalize = p.normalize;
    a.map_dtype = p.map_dtype;
    a.variant = p.variant;
    a.fused = fused;
    a.crossing = crossing;
    for (int k = 0; k < n_views; ++k) a.xf[k] = compose(in_cams[k], *target);
    const size_t elem = p.map_dtype == GVS_F16 ? 4 : 8;  // half2 or float2 (d, omega)
    for (int k = 0; k < n_views; ++k) a.vb[k] = reinterpret_cast<const char *>(a.dw) + (size_t)k * W * H * elem;
    return a;
}

}  // namespace

extern "C" {

gvs_status gvs_weight_map(const void *in_depths, int32_t depth_dtype, int32_t n_views, int32_t width,
                          int32_t height, float mu, float weight_const, int32_t window, int32_t map_dtype, void *map,
                          size_t map_bytes, void *stream) {
    const Range nvtx_range("gvs_weight_map");
    if (n_views < 0 || n_views > GVS_MAX_VIEWS) return fail(GVS_ERR_INVALID_ARG, "weight map: n_views out of range");
    if (width < 1 || height < 1 || width > GVS_MAX_DIM || height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "weight map: image size out of range");
    gvs_status s = check_weight_params(mu, weight_const, window);
    if (s != GVS_OK) return s;
    if (depth_dtype != GVS_F32 && depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "weight map: depth_dtype must be GVS_F32 or GVS_F16");
    if (map_dtype != GVS_F32 && map_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "weight map: map_dtype must be GVS_F32 or GVS_F16");
    if (n_views == 0) return GVS_OK;
    if (!in_depths || !aligned(in_depths, 16)) return fail(GVS_ERR_INVALID_ARG, "weight map: in_depths is NULL or misaligned");
    const size_t need = gvs_fuse_workspace_bytes(n_views, width, height);
    if (!map || map_bytes < need || !aligned(map, 256))
        return fail(GVS_ERR_WORKSPACE, "weight map: map needs %zu bytes, 256-byte aligned", need);
    cudaError_t e = gvs::launch_weight_map(in_depths, depth_dtype, map, map_dtype, n_views, width, height, mu,
                                           weight_const, window, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "weight map launch");
    return GVS_OK;
}

gvs_status gvs_fuse_depth_from_map(const gvs_camera *in_cams, const void *map, size_t map_bytes, int32_t n_views,
                                   const gvs_camera *target, const gvs_fuse_params *params, float *fused_depth,
                                   int16_t *crossing, void *stream) {
    const Range nvtx_range("gvs_fuse_depth_from_map");
    int32_t W = 0, H = 0;
    gvs_status s = check_fuse_common(in_cams, n_views, target, params, fused_depth, crossing, &W, &H);
    if (s != GVS_OK) return s;
    const size_t need = gvs_fuse_workspace_bytes(n_views, W, H);
    if (n_views > 0 && (!map || map_bytes < need || !aligned(map, 256)))
        return fail(GVS_ERR_WORKSPACE, "fuse: map needs %zu bytes, 256-byte aligned", need);
    gvs::FuseArgs a = fuse_args(in_cams, map, n_views, W, H, target, *params, fused_depth, crossing);
    cudaError_t e = gvs::launch_fuse(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fuse: launch");
    return GVS_OK;
}

gvs_status gvs_fuse_depth_temporal(const gvs_camera *in_cams, const void *map, size_t map_bytes, int32_t n_views,
                                   const gvs_camera *target, const gvs_fuse_params *params, const float *prev_depth,
                                   const float *w_tmp, float *fused_depth, int16_t *crossing, float *view_weight,
                                   void *stream) {
    const Range nvtx_range("gvs_fuse_depth_temporal");
    int32_t W = 0, H = 0;
    gvs_status s = check_fuse_common(in_cams, n_views, target, params, fused_depth, crossing, &W, &H);
    if (s != GVS_OK) return s;
    if (!prev_depth || !w_tmp || !aligned(prev_depth, 16) || !aligned(w_tmp, 16) ||
        (view_weight && !aligned(view_weight, 16)))
        return fail(GVS_ERR_INVALID_ARG, "fuse temporal: prev_depth and w_tmp required, 16-byte aligned");
    const size_t need = gvs_fuse_workspace_bytes(n_views, W, H);
    if (n_views > 0 && (!map || map_bytes < need || !aligned(map, 256)))
        return fail(GVS_ERR_WORKSPACE, "fuse temporal: map needs %zu bytes, 256-byte aligned", need);
    gvs::FuseArgs a = fuse_args(in_cams, map, n_views, W, H, target, *params, fused_depth, crossing);
    a.tmp_depth = prev_depth;
    a.tmp_weight = w_tmp;
    a.wview = view_weight;
    cudaError_t e = gvs::launch_fuse(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fuse temporal: launch");
    return GVS_OK;
}

gvs_status gvs_temporal_weight(const void *masks, int32_t mask_dtype, const int32_t *winner, int32_t n_views,
                               int32_t width, int32_t height, int32_t target_width, int32_t target_height,
                               const float *w_tmp_prev, const float *w_view_prev, float beta_t, float eta,
                               float *w_tmp, float *target_mask, void *stream) {
    const Range nvtx_range("gvs_temporal_weight");
    if (n_views < 0 || n_views > GVS_MAX_VIEWS || width < 1 || height < 1 || target_width < 1 || target_height < 1 ||
        width > GVS_MAX_DIM || height > GVS_MAX_DIM || target_width > GVS_MAX_DIM || target_height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "temporal weight: sizes out of range");
    if (mask_dtype != GVS_F32 && mask_dtype != GVS_U8)
        return fail(GVS_ERR_UNSUPPORTED, "temporal weight: mask_dtype must be GVS_F32 or GVS_U8");
    if (!(isfinite(beta_t) && beta_t >= 0.0f) || !(isfinite(eta) && eta >= 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "temporal weight: beta_t and eta must be finite and >= 0");
    if ((n_views > 0 && (!masks || !winner)) || !w_tmp_prev || !w_view_prev || !w_tmp)
        return fail(GVS_ERR_INVALID_ARG, "temporal weight: NULL array");
    cudaError_t e = gvs::launch_temporal_weight(masks, mask_dtype, winner, n_views, (int64_t)width * height,
                                                (int64_t)target_width * target_height, w_tmp_prev, w_view_prev,
                                                beta_t, eta, w_tmp, target_mask, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "temporal weight: launch");
    return GVS_OK;
}

gvs_status gvs_guided_mask(const float *warped_depth, const uint8_t *alpha, const float *fused_depth,
                           int32_t n_views, int32_t target_width, int32_t target_height, float mu_guide,
                           uint8_t *guided, void *stream) {
    const Range nvtx_range("gvs_guided_mask");
    if (n_views < 0 || n_views > GVS_MAX_VIEWS || target_width < 1 || target_height < 1)
        return fail(GVS_ERR_INVALID_ARG, "guided mask: sizes out of range");
    if (!(isfinite(mu_guide) && mu_guide >= 0.0f)) return fail(GVS_ERR_INVALID_ARG, "guided mask: mu_guide must be >= 0");
    if (n_views == 0) return GVS_OK;
    if (!warped_depth || !alpha || !fused_depth || !guided) return fail(GVS_ERR_INVALID_ARG, "guided mask: NULL array");
    cudaError_t e = gvs::launch_guided_mask(warped_depth, alpha, fused_depth, n_views,
                                            (int64_t)target_width * target_height, mu_guide, guided,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "guided mask: launch");
    return GVS_OK;
}

gvs_status gvs_fuse_depth(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                          const gvs_camera *target, const gvs_fuse_params *params, float *fused_depth,
                          int16_t *crossing, void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_fuse_depth");
    int32_t W = 0, H = 0;
    gvs_status s = check_fuse_common(in_cams, n_views, target, params, fused_depth, crossing, &W, &H);
    if (s != GVS_OK) return s;
    s = check_weight_params(params->mu, params->weight_const, params->window);
    if (s != GVS_OK) return s;
    if (n_views > 0 && (!in_depths || !aligned(in_depths, 16)))
        return fail(GVS_ERR_INVALID_ARG, "fuse: in_depths is NULL or not 16-byte aligned");
    const size_t need = gvs_fuse_workspace_bytes(n_views, W, H);
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned(workspace, 256)))
        return fail(GVS_ERR_WORKSPACE, "fuse: workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = gvs::launch_weight_map(in_depths, params->depth_dtype, workspace, params->map_dtype, n_views, W,
                                           H, params->mu, params->weight_const, params->window, st);
    if (e != cudaSuccess) return cuda_fail(e, "fuse: weight map launch");
    gvs::FuseArgs a = fuse_args(in_cams, workspace, n_views, W, H, target, *params, fused_depth, crossing);
    e = gvs::launch_fuse(a, st);
    if (e != cudaSuccess) return cuda_fail(e, "fuse: launch");
    return GVS_OK;
}

size_t gvs_fuse_backward_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
    if (n_views < 0 || width < 0 || height < 0) return 0;
    return align_up((size_t)n_views * (size_t)width * (size_t)height * sizeof(float2), 256);
}

gvs_status gvs_fuse_depth_backward(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                                   const gvs_camera *target, const gvs_fuse_params *params, const void *map,
                                   size_t map_bytes, const int16_t *crossing, const float *grad_fused,
                                   float *grad_depths, void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_fuse_depth_backward");
    int32_t W = 0, H = 0;
    // the checks of the forward, with the fused-depth output replaced by its gradient
    gvs_status s = check_fuse_common(in_cams, n_views, target, params, grad_fused, crossing, &W, &H);
    if (s != GVS_OK) return s;
    s = check_weight_params(params->mu, params->weight_const, params->window);
    if (s != GVS_OK) return s;
    if (params->normalize != 0)
        return fail(GVS_ERR_UNSUPPORTED, "fuse backward: only the unnormalised sum (normalize = 0) is differentiated");
    if (!crossing) return fail(GVS_ERR_INVALID_ARG, "fuse backward: crossing (from the forward) is NULL");
    if (n_views == 0) return GVS_OK;
    if (!in_depths || !aligned(in_depths, 16) || !grad_depths || !aligned(grad_depths, 16))
        return fail(GVS_ERR_INVALID_ARG, "fuse backward: in_depths / grad_depths NULL or not 16-byte aligned");
    const size_t need_map = gvs_fuse_workspace_bytes(n_views, W, H);
    if (!map || map_bytes < need_map || !aligned(map, 256))
        return fail(GVS_ERR_WORKSPACE, "fuse backward: map needs %zu bytes, 256-byte aligned", need_map);
    const size_t need = gvs_fuse_backward_workspace_bytes(n_views, W, H);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "fuse backward: workspace needs %zu bytes, 256-byte aligned", need);
    gvs::FuseArgs a = fuse_args(in_cams, map, n_views, W, H, target, *params, grad_depths, nullptr);
    cudaError_t e = gvs::launch_fuse_backward(a, in_depths, params->depth_dtype, crossing, grad_fused, grad_depths,
                                              reinterpret_cast<float2 *>(workspace), params->mu,
                                              params->weight_const, params->window, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fuse backward: launch");
    return GVS_OK;
}

size_t gvs_splat_workspace_bytes(int32_t n_views, int32_t target_width, int32_t target_height) {
    (void)n_views;
    if (target_width < 0 || target_height < 0) return 0;
    return align_up((size_t)target_width * (size_t)target_height * sizeof(unsigned long long), 256);
}

gvs_status gvs_forward_splat(const gvs_camera *in_cams, const void *in_depths, const uint32_t *in_rgba,
                             int32_t n_views, const gvs_camera *target, const gvs_splat_params *params,
                             const float *fused_depth, int32_t *winner, uint32_t *warped_rgba, float *warped_depth,
                             uint8_t *alpha, uint8_t *guided, void *workspace, size_t workspace_bytes,
                             void *stream) {
    const Range nvtx_range("gvs_forward_splat");
    int32_t W = 0, H = 0;
    if (!params) return fail(GVS_ERR_INVALID_ARG, "splat: params is NULL");
    if (!views_ok(in_cams, n_views, &W, &H))
        return fail(GVS_ERR_INVALID_ARG, "splat: input cameras invalid, of different sizes, or n_views out of range");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "splat: target camera invalid");
    const gvs_splat_params &p = *params;
    if (p.footprint != 0 && p.footprint != 1) return fail(GVS_ERR_INVALID_ARG, "splat: footprint must be 0 or 1");
    if (p.depth_dtype != GVS_F32 && p.depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "splat: depth_dtype must be GVS_F32 or GVS_F16");
    if (!(isfinite(p.max_half_width) && p.max_half_width >= 0.5f && p.max_half_width <= 64.0f))
        return fail(GVS_ERR_INVALID_ARG, "splat: max_half_width must be in [0.5, 64]");
    if (guided && !(isfinite(p.mu_guide) && p.mu_guide >= 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "splat: mu_guide must be >= 0");
    if (guided && !fused_depth) return fail(GVS_ERR_INVALID_ARG, "splat: guided mask needs fused_depth");
    if (p.guide_reject != 0 && p.guide_reject != 1)
        return fail(GVS_ERR_INVALID_ARG, "splat: guide_reject must be 0 or 1");
    if (p.guide_reject && !fused_depth) return fail(GVS_ERR_INVALID_ARG, "splat: guide_reject needs fused_depth");
    if (p.guide_reject && !(isfinite(p.mu_guide) && p.mu_guide >= 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "splat: mu_guide must be >= 0");
    if (n_views == 0) return GVS_OK;
    if (!in_depths || !in_rgba || !winner) return fail(GVS_ERR_INVALID_ARG, "splat: NULL array");
    const void *arrs[] = {in_depths, in_rgba, fused_depth, winner, warped_rgba, warped_depth, alpha, guided};
    for (const void *q : arrs)
        if (q && !aligned(q, 16)) return fail(GVS_ERR_INVALID_ARG, "splat: arrays must be 16-byte aligned");
    const size_t slot = gvs_splat_workspace_bytes(n_views, target->width, target->height);
    if (!workspace || workspace_bytes < slot || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "splat: workspace needs at least %zu bytes, 256-byte aligned", slot);

    gvs::SplatArgs a;
    memset(&a, 0, sizeof(a));
    a.depth = in_depths;
    a.depth_dtype = p.depth_dtype;
    a.rgba = in_rgba;
    a.W = W;
    a.H = H;
    a.Wt = target->width;
    a.Ht = target->height;
    a.footprint = p.footprint;
    a.guide_reject = p.guide_reject;
    a.max_hw = p.max_half_width;
    a.mu_guide = p.mu_guide;
    a.fused = fused_depth;
    a.winner = winner;
    a.warped_rgba = warped_rgba;
    a.warped_depth = warped_depth;
    a.alpha = alpha;
    a.guided = guided;
    a.keys = reinterpret_cast<unsigned long long *>(workspace);
    const size_t slot_keys = (size_t)target->width * target->height * sizeof(unsigned long long);
    size_t slots = workspace_bytes / slot_keys;
    a.slots = (int)(slots > (size_t)n_views ? (size_t)n_views : slots);
    for (int k = 0; k < n_views; ++k) {
        a.v[k].xf = compose(*target, in_cams[k]);
        a.v[k].f_ratio = (float)(target->fx / in_cams[k].fx);
    }
    cudaError_t e = gvs::launch_splat(a, n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "splat: launch");
    return GVS_OK;
}

}  // extern "C"

namespace {

// Slots of (keys, accumulators) that fit a soft-splat workspace: keys for all
// slots first, then the float4 accumulators from the next 256-byte boundary.
int soft_slots(size_t ws_bytes, int64_t HWt, int K) {
    int slots = 0;
    for (int s = 1; s <= K; ++s) {
        const size_t need = align_up((size_t)s * HWt * 8, 256) + (size_t)s * HWt * 16;
        if (need > ws_bytes) break;
        slots = s;
    }
    return slots;
}

gvs_status soft_common(const gvs_camera *in_cams, const void *in_depths, const void *in_color, int32_t n_views,
                       const gvs_camera *target, const gvs_soft_splat_params *params, gvs::SplatArgs *a) {
    int32_t W = 0, H = 0;
    if (!params) return fail(GVS_ERR_INVALID_ARG, "soft splat: params is NULL");
    if (!views_ok(in_cams, n_views, &W, &H))
        return fail(GVS_ERR_INVALID_ARG, "soft splat: input cameras invalid, of different sizes, or n_views out of range");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "soft splat: target camera invalid");
    const gvs_soft_splat_params &p = *params;
    if (!(isfinite(p.max_half_width) && p.max_half_width >= 0.5f && p.max_half_width <= 64.0f))
        return fail(GVS_ERR_INVALID_ARG, "soft splat: max_half_width must be in [0.5, 64]");
    if (!(isfinite(p.mu_band) && p.mu_band >= 0.0f)) return fail(GVS_ERR_INVALID_ARG, "soft splat: mu_band must be >= 0");
    if (p.depth_dtype != GVS_F32 && p.depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "soft splat: depth_dtype must be GVS_F32 or GVS_F16");
    if (p.color_dtype != GVS_F32 && p.color_dtype != GVS_BF16)
        return fail(GVS_ERR_UNSUPPORTED, "soft splat: color_dtype must be GVS_F32 or GVS_BF16");
    if (n_views > 0 && (!in_depths || !in_color || !aligned(in_depths, 16) || !aligned(in_color, 16)))
        return fail(GVS_ERR_INVALID_ARG, "soft splat: inputs NULL or not 16-byte aligned");
    memset(a, 0, sizeof(*a));
    a->depth = in_depths;
    a->depth_dtype = p.depth_dtype;
    a->color = in_color;
    a->color_dtype = p.color_dtype;
    a->W = W;
    a->H = H;
    a->Wt = target->width;
    a->Ht = target->height;
    a->footprint = 1;
    a->max_hw = p.max_half_width;
    a->mu_band = p.mu_band;
    for (int k = 0; k < n_views; ++k) {
        a->v[k].xf = compose(*target, in_cams[k]);
        a->v[k].f_ratio = (float)(target->fx / in_cams[k].fx);
    }
    return GVS_OK;
}

}  // namespace

extern "C" {

size_t gvs_soft_splat_workspace_bytes(int32_t n_views, int32_t target_width, int32_t target_height) {
    (void)n_views;
    if (target_width < 0 || target_height < 0) return 0;
    const size_t HWt = (size_t)target_width * target_height;
    return align_up(align_up(HWt * 8, 256) + HWt * 16, 256);
}

gvs_status gvs_soft_splat(const gvs_camera *in_cams, const void *in_depths, const void *in_color, int32_t n_views,
                          const gvs_camera *target, const gvs_soft_splat_params *params, int32_t *winner,
                          float *warped_color, float *warped_depth, float *weight_sum, uint8_t *alpha,
                          void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_soft_splat");
    gvs::SplatArgs a;
    gvs_status s = soft_common(in_cams, in_depths, in_color, n_views, target, params, &a);
    if (s != GVS_OK) return s;
    if (n_views == 0) return GVS_OK;
    const void *outs[] = {winner, warped_color, weight_sum};
    for (const void *q : outs)
        if (!q || !aligned(q, 16)) return fail(GVS_ERR_INVALID_ARG, "soft splat: winner, warped_color and weight_sum are required, 16-byte aligned");
    if ((warped_depth && !aligned(warped_depth, 16)) || (alpha && !aligned(alpha, 16)))
        return fail(GVS_ERR_INVALID_ARG, "soft splat: outputs must be 16-byte aligned");
    const int64_t HWt = (int64_t)target->width * target->height;
    const int slots = soft_slots(workspace_bytes, HWt, n_views);
    if (!workspace || !aligned(workspace, 256) || slots < 1)
        return fail(GVS_ERR_WORKSPACE, "soft splat: workspace needs %zu bytes, 256-byte aligned",
                    gvs_soft_splat_workspace_bytes(n_views, target->width, target->height));
    a.keys = reinterpret_cast<unsigned long long *>(workspace);
    a.acc = reinterpret_cast<float4 *>(reinterpret_cast<char *>(workspace) + align_up((size_t)slots * HWt * 8, 256));
    a.slots = slots;
    a.winner = winner;
    a.out_color = reinterpret_cast<float4 *>(warped_color);
    a.warped_depth = warped_depth;
    a.wsum = weight_sum;
    a.alpha = alpha;
    cudaError_t e = gvs::launch_soft_splat(a, n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "soft splat: launch");
    return GVS_OK;
}

gvs_status gvs_soft_splat_backward(const gvs_camera *in_cams, const void *in_depths, const void *in_color,
                                   int32_t n_views, const gvs_camera *target, const gvs_soft_splat_params *params,
                                   const int32_t *winner, const float *warped_color, const float *warped_depth,
                                   const float *weight_sum, const float *grad_color, const float *grad_depth,
                                   float *grad_in_depth, float *grad_in_color, void *stream) {
    const Range nvtx_range("gvs_soft_splat_backward");
    gvs::SplatArgs a;
    gvs_status s = soft_common(in_cams, in_depths, in_color, n_views, target, params, &a);
    if (s != GVS_OK) return s;
    if (n_views == 0) return GVS_OK;
    const void *req[] = {winner, warped_color, warped_depth, weight_sum, grad_color, grad_in_depth, grad_in_color};
    for (const void *q : req)
        if (!q || !aligned(q, 16)) return fail(GVS_ERR_INVALID_ARG, "soft splat backward: NULL or misaligned array");
    if (grad_depth && !aligned(grad_depth, 16)) return fail(GVS_ERR_INVALID_ARG, "soft splat backward: grad_depth misaligned");
    a.winner = const_cast<int32_t *>(winner);
    a.out_color = const_cast<float4 *>(reinterpret_cast<const float4 *>(warped_color));
    a.warped_depth = const_cast<float *>(warped_depth);
    a.wsum = const_cast<float *>(weight_sum);
    a.grad_color = reinterpret_cast<const float4 *>(grad_color);
    a.grad_depth = grad_depth;
    a.grad_in_depth = grad_in_depth;
    a.grad_in_color = reinterpret_cast<float4 *>(grad_in_color);
    cudaError_t e = gvs::launch_soft_splat_backward(a, n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "soft splat backward: launch");
    return GVS_OK;
}

gvs_status gvs_soft_splat_backward_blended(const gvs_camera *in_cams, const void *in_depths, const void *in_color,
                                           int32_t n_views, const gvs_camera *target,
                                           const gvs_soft_splat_params *params, const int32_t *winner,
                                           const float *warped_color, const float *warped_depth,
                                           const float *weight_sum, const float *grad_pixel, float *grad_in_depth,
                                           float *grad_in_color, void *stream) {
    const Range nvtx_range("gvs_soft_splat_backward_blended");
    gvs::SplatArgs a;
    gvs_status s = soft_common(in_cams, in_depths, in_color, n_views, target, params, &a);
    if (s != GVS_OK) return s;
    if (n_views == 0) return GVS_OK;
    const void *req[] = {winner, warped_color, warped_depth, weight_sum, grad_pixel, grad_in_depth, grad_in_color};
    for (const void *q : req)
        if (!q || !aligned(q, 16))
            return fail(GVS_ERR_INVALID_ARG, "soft splat backward (blended): NULL or misaligned array");
    a.winner = const_cast<int32_t *>(winner);
    a.out_color = const_cast<float4 *>(reinterpret_cast<const float4 *>(warped_color));
    a.warped_depth = const_cast<float *>(warped_depth);
    a.wsum = const_cast<float *>(weight_sum);
    a.grad_pixel = reinterpret_cast<const float4 *>(grad_pixel);
    a.grad_in_depth = grad_in_depth;
    a.grad_in_color = reinterpret_cast<float4 *>(grad_in_color);
    cudaError_t e = gvs::launch_soft_splat_backward(a, n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "soft splat backward (blended): launch");
    return GVS_OK;
}

size_t gvs_uniform_blend_loss_workspace_bytes(int32_t target_width, int32_t target_height) {
    if (target_width < 1 || target_height < 1 || target_width > GVS_MAX_DIM || target_height > GVS_MAX_DIM) return 0;
    return gvs::blend_loss_layout((int64_t)target_width * target_height).total;
}

gvs_status gvs_uniform_blend_loss(int32_t n_views, int32_t target_width, int32_t target_height,
                                  const float *warped_color, const uint8_t *alpha, const float *warped_depth,
                                  const float *fused_depth, const float *ground_truth, float w_l1, float w_depth,
                                  double *loss, float *grad_pixel, float *grad_fused, void *workspace,
                                  size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_uniform_blend_loss");
    if (n_views < 1 || n_views > GVS_MAX_VIEWS)
        return fail(GVS_ERR_INVALID_ARG, "blend loss: n_views must be in [1, %d]", GVS_MAX_VIEWS);
    if (target_width < 1 || target_height < 1 || target_width > GVS_MAX_DIM || target_height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "blend loss: target size out of range");
    if (!(isfinite(w_l1) && w_l1 >= 0.0f && isfinite(w_depth) && w_depth >= 0.0f))
        return fail(GVS_ERR_INVALID_ARG, "blend loss: weights must be finite and >= 0");
    if (!warped_color || !aligned(warped_color, 16) || !alpha || !warped_depth || !aligned(warped_depth, 4) ||
        !fused_depth || !aligned(fused_depth, 4) || !ground_truth || !aligned(ground_truth, 4) || !loss ||
        !aligned(loss, 8))
        return fail(GVS_ERR_INVALID_ARG, "blend loss: NULL or misaligned input or loss");
    if ((grad_pixel && !aligned(grad_pixel, 16)) || (grad_fused && !aligned(grad_fused, 4)))
        return fail(GVS_ERR_INVALID_ARG, "blend loss: misaligned gradient output");
    const int64_t HWt = (int64_t)target_width * target_height;
    const size_t need = gvs::blend_loss_layout(HWt).total;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "blend loss: workspace needs %zu bytes, 256-byte aligned", need);
    cudaError_t e = gvs::launch_blend_loss(n_views, HWt, reinterpret_cast<const float4 *>(warped_color), alpha,
                                           warped_depth, fused_depth, ground_truth, w_l1, w_depth, loss,
                                           reinterpret_cast<float4 *>(grad_pixel), grad_fused,
                                           reinterpret_cast<char *>(workspace), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend loss: launch");
    return GVS_OK;
}

gvs_status gvs_uniform_blend_loss_grad(int32_t target_width, int32_t target_height, const float *grad_loss,
                                       float *grad_pixel, float *grad_fused, const void *workspace,
                                       size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_uniform_blend_loss_grad");
    if (target_width < 1 || target_height < 1 || target_width > GVS_MAX_DIM || target_height > GVS_MAX_DIM)
        return fail(GVS_ERR_INVALID_ARG, "blend loss gradient: target size out of range");
    if (!grad_pixel && !grad_fused)
        return fail(GVS_ERR_INVALID_ARG, "blend loss gradient: no output");
    if ((grad_pixel && !aligned(grad_pixel, 16)) || (grad_fused && !aligned(grad_fused, 4)) ||
        (grad_loss && !aligned(grad_loss, 4)))
        return fail(GVS_ERR_INVALID_ARG, "blend loss gradient: misaligned array");
    const int64_t HWt = (int64_t)target_width * target_height;
    const size_t need = gvs::blend_loss_layout(HWt).total;
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "blend loss gradient: workspace needs %zu bytes, 256-byte aligned", need);
    cudaError_t e = gvs::launch_blend_loss_grad(HWt, reinterpret_cast<const char *>(workspace), grad_loss,
                                                reinterpret_cast<float4 *>(grad_pixel), grad_fused,
                                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend loss gradient: launch");
    return GVS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward splat without any device allocation.
//
// Some callers cannot hand the library a workspace: a plugin inside a host
// application that owns every device allocation through its own allocator,
// code recorded into a CUDA graph where a cudaMalloc would break the capture,
// or a real-time loop that must not block on the allocator (cudaMalloc and
// cudaFree can synchronize the device).  For them the z-buffer lives in a
// file-scope device array, loaded with the library and held by every GPU that
// loads it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocKeys = size_t(1) << 21;  // 16 MiB of 64-bit keys: targets up to 2,097,152 pixels
static __device__ __align__(256) unsigned long long g_noalloc_keys[kNoAllocKeys];

// Device address of g_noalloc_keys in the calling thread's current CUDA
// context.  In host code the symbol is only a host-side handle, never a device
// address, so it must not be passed to a kernel directly.  A module, and with
// it the array, is loaded per context: the primary context of a device, a
// context a host application created itself, or the primary context created
// again after a cudaDeviceReset each have their own copy at their own address.
// The lookup is therefore cached per context, keyed by the driver's context id
// (unique for the life of the process, never reused), not by device ordinal.
// The two driver calls are fetched through the runtime, so the library does not
// link the driver library itself.
typedef int (*ctx_get_current_fn)(void **ctx);
typedef int (*ctx_get_id_fn)(void *ctx, unsigned long long *id);

bool current_context_id(unsigned long long *id) {
    static std::once_flag once;
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_get_id_fn>(f);
    });
    if (!get_current || !get_id) return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

unsigned long long *noalloc_keys_on_current_context(gvs_status *st) {
    constexpr int kSlots = 64;
    static std::mutex mu;
    static unsigned long long ids[kSlots] = {0};
    static unsigned long long *addr[kSlots] = {nullptr};
    static int next = 0;
    unsigned long long id = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!current_context_id(&id)) {
        // no context is current yet: the runtime binds the device's primary
        // context on its first call, so look the array up (which does that) and ask again
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_keys);
        if (e != cudaSuccess || !p) {
            *st = fail(GVS_ERR_CUDA, "splat (no-alloc): cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return nullptr;
        }
        if (!current_context_id(&id)) {
            *st = fail(GVS_ERR_DEVICE, "splat (no-alloc): cannot identify the current CUDA context");
            return nullptr;
        }
    }
    for (int i = 0; i < kSlots; ++i)
        if (addr[i] && ids[i] == id) {
            *st = GVS_OK;
            return addr[i];
        }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_keys);
    if (e != cudaSuccess || !p) {
        *st = fail(GVS_ERR_CUDA, "splat (no-alloc): cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return nullptr;
    }
    // a context destroyed since keeps its entry until it is the oldest of kSlots others
    ids[next] = id;
    addr[next] = reinterpret_cast<unsigned long long *>(p);
    next = (next + 1) % kSlots;
    *st = GVS_OK;
    return reinterpret_cast<unsigned long long *>(p);
}

}  // namespace

extern "C" gvs_status gvs_forward_splat_noalloc(const gvs_camera *in_cams, const void *in_depths,
                                                const uint32_t *in_rgba, int32_t n_views, const gvs_camera *target,
                                                const gvs_splat_params *params, const float *fused_depth,
                                                int32_t *winner, uint32_t *warped_rgba, float *warped_depth,
                                                uint8_t *alpha, uint8_t *guided, void *stream) {
    if (!target) return fail(GVS_ERR_INVALID_ARG, "splat (no-alloc): target camera is NULL");
    const int64_t pixels = (int64_t)target->width * (int64_t)target->height;
    if (pixels > (int64_t)kNoAllocKeys)
        return fail(GVS_ERR_INVALID_ARG,
                    "splat (no-alloc): target has %lld pixels; this entry point holds a z-buffer for at most %zu",
                    (long long)pixels, kNoAllocKeys);
    gvs_status st = GVS_OK;
    unsigned long long *keys = noalloc_keys_on_current_context(&st);
    if (!keys) return st;
    return gvs_forward_splat(in_cams, in_depths, in_rgba, n_views, target, params, fused_depth, winner,
                             warped_rgba, warped_depth, alpha, guided, keys, kNoAllocKeys * sizeof(unsigned long long),
                             stream);
}

// ---------------------------------------------------------------------------
// Batched fusion: many (frame, target) items, one persistent launch.
// ---------------------------------------------------------------------------
struct gvs_fuse_batch {
    int K, map_dtype, variant, n_items, total;
    gvs::BatchItem *d_items;
    unsigned *d_counter;
};

extern "C" {

size_t gvs_fuse_batch_bytes(int32_t n_items) {
    if (n_items < 0) return 0;
    return align_up((size_t)n_items * sizeof(gvs::BatchItem), 256) + 256;
}

gvs_status gvs_fuse_batch_create(const gvs_camera *in_cams, int32_t n_views, const gvs_fuse_item *items,
                                 int32_t n_items, const gvs_fuse_params *params, void *table, size_t table_bytes,
                                 gvs_fuse_batch **out) {
    const Range nvtx_range("gvs_fuse_batch_create");
    if (!out) return fail(GVS_ERR_INVALID_ARG, "fuse batch: out is NULL");
    *out = nullptr;
    if (n_items < 1 || n_items > GVS_MAX_BATCH_ITEMS || !items)
        return fail(GVS_ERR_INVALID_ARG, "fuse batch: n_items must be in [1, %d]", GVS_MAX_BATCH_ITEMS);
    if (n_views < 1) return fail(GVS_ERR_INVALID_ARG, "fuse batch: needs at least one input view");
    const size_t need = gvs_fuse_batch_bytes(n_items);
    if (!table || table_bytes < need || !aligned(table, 256))
        return fail(GVS_ERR_WORKSPACE, "fuse batch: table needs %zu bytes, 256-byte aligned", need);
    std::vector<gvs::BatchItem> host((size_t)n_items);
    int64_t total = 0;
    int32_t W = 0, H = 0;
    for (int i = 0; i < n_items; ++i) {
        const gvs_fuse_item &it = items[i];
        gvs_status s = check_fuse_common(in_cams, n_views, it.target, params, it.fused_depth, it.crossing, &W, &H);
        if (s != GVS_OK) return s;
        const size_t need_map = gvs_fuse_workspace_bytes(n_views, W, H);
        if (!it.map || it.map_bytes < need_map || !aligned(it.map, 256))
            return fail(GVS_ERR_WORKSPACE, "fuse batch: item %d map needs %zu bytes, 256-byte aligned", i, need_map);
        host[i].args = fuse_args(in_cams, it.map, n_views, W, H, it.target, *params, it.fused_depth, it.crossing);
        host[i].bundle_begin = (int)total;
        total += gvs::bundle_count(it.target->width, it.target->height, n_views, params->variant);
        if (total > INT32_MAX / 2) return fail(GVS_ERR_UNSUPPORTED, "fuse batch: too many target pixels");
    }
    cudaError_t e = cudaMemcpy(table, host.data(), host.size() * sizeof(gvs::BatchItem), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "fuse batch: copying the item table");
    gvs_fuse_batch *b = new (std::nothrow) gvs_fuse_batch;
    if (!b) return fail(GVS_ERR_INVALID_ARG, "fuse batch: out of host memory");
    b->K = n_views;
    b->map_dtype = params->map_dtype;
    b->variant = params->variant;
    b->n_items = n_items;
    b->total = (int)total;
    b->d_items = reinterpret_cast<gvs::BatchItem *>(table);
    b->d_counter = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(table) +
                                                align_up((size_t)n_items * sizeof(gvs::BatchItem), 256));
    *out = b;
    return GVS_OK;
}

gvs_status gvs_fuse_batch_launch(const gvs_fuse_batch *b, void *stream) {
    const Range nvtx_range("gvs_fuse_batch_launch");
    if (!b) return fail(GVS_ERR_INVALID_ARG, "fuse batch: NULL batch");
    cudaError_t e = gvs::launch_fuse_batch(b->d_items, b->n_items, b->total, b->d_counter, b->K, b->map_dtype,
                                           b->variant, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fuse batch: launch");
    return GVS_OK;
}

void gvs_fuse_batch_destroy(gvs_fuse_batch *b) { delete b; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Pixel-sized Gaussian forward render (Sec. 3.1, Supplement A.3).
// ---------------------------------------------------------------------------
extern "C" {

size_t gvs_gauss_splat_workspace_bytes(int32_t width, int32_t height, int32_t target_width, int32_t target_height,
                                       int32_t max_radius) {
    if (width < 1 || height < 1 || target_width < 1 || target_height < 1 || max_radius < 1 ||
        max_radius > GVS_MAX_GAUSS_RADIUS)
        return 0;
    return gvs::gauss_layout(width, height, target_width, target_height, max_radius).total;
}

gvs_status gvs_gauss_splat(const gvs_camera *in_cams, const void *in_depths, const uint32_t *in_rgba,
                           int32_t n_views, const gvs_camera *target, const gvs_gauss_params *params, float *color,
                           float *depth, void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_gauss_splat");
    int32_t W = 0, H = 0;
    if (!params) return fail(GVS_ERR_INVALID_ARG, "gauss splat: params is NULL");
    if (!views_ok(in_cams, n_views, &W, &H))
        return fail(GVS_ERR_INVALID_ARG, "gauss splat: input cameras invalid, of different sizes, or n_views out of range");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "gauss splat: target camera invalid");
    const gvs_gauss_params &p = *params;
    if (!(isfinite(p.scale_px) && p.scale_px > 0.0f && p.scale_px <= 16.0f))
        return fail(GVS_ERR_INVALID_ARG, "gauss splat: scale_px must be in (0, 16]");
    if (p.max_radius < 1 || p.max_radius > GVS_MAX_GAUSS_RADIUS)
        return fail(GVS_ERR_INVALID_ARG, "gauss splat: max_radius must be in [1, %d]", GVS_MAX_GAUSS_RADIUS);
    if (p.depth_dtype != GVS_F32 && p.depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "gauss splat: depth_dtype must be GVS_F32 or GVS_F16");
    if (n_views == 0) return GVS_OK;
    if (!in_depths || !in_rgba || !color || !depth) return fail(GVS_ERR_INVALID_ARG, "gauss splat: NULL array");
    const void *arrs[] = {in_depths, in_rgba, color, depth};
    for (const void *q : arrs)
        if (!aligned(q, 16)) return fail(GVS_ERR_INVALID_ARG, "gauss splat: arrays must be 16-byte aligned");
    const size_t need = gvs_gauss_splat_workspace_bytes(W, H, target->width, target->height, p.max_radius);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "gauss splat: workspace needs at least %zu bytes, 256-byte aligned", need);
    gvs::GaussArgs a;
    memset(&a, 0, sizeof(a));
    a.depth = in_depths;
    a.depth_dtype = p.depth_dtype;
    a.rgba = in_rgba;
    a.W = W;
    a.H = H;
    a.Wt = target->width;
    a.Ht = target->height;
    a.scale_px = p.scale_px;
    a.max_radius = p.max_radius;
    a.in32[0] = (float)target->fx;
    a.in32[1] = (float)target->fy;
    a.in32[2] = (float)target->cx;
    a.in32[3] = (float)target->cy;
    a.in32[4] = (float)(target->fy / target->fx);
    a.color = reinterpret_cast<float4 *>(color);
    a.depth_out = depth;
    a.ws = reinterpret_cast<char *>(workspace);
    a.L = gvs::gauss_layout(W, H, target->width, target->height, p.max_radius);
    for (int k = 0; k < n_views; ++k) {
        a.xf[k] = compose(*target, in_cams[k]);
        a.f_ratio[k] = (float)(target->fx / in_cams[k].fx);
    }
    cudaError_t e = gvs::launch_gauss_splat(a, n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gauss splat: launch");
    return GVS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Blending-network input and blend (Sec. 3.3).
// ---------------------------------------------------------------------------
namespace {

bool blend_common(int32_t n_views, int32_t Wt, int32_t Ht, const uint32_t *warped_rgba, const float *warped_depth,
                  const uint8_t *alpha, const float *fused_depth, const char *what, gvs_status *st) {
    if (n_views < 1 || n_views > GVS_MAX_VIEWS || Wt < 1 || Ht < 1 || Wt > GVS_MAX_DIM || Ht > GVS_MAX_DIM) {
        *st = fail(GVS_ERR_INVALID_ARG, "%s: n_views or target size out of range", what);
        return false;
    }
    if (!warped_rgba || !warped_depth || !alpha || !fused_depth) {
        *st = fail(GVS_ERR_INVALID_ARG, "%s: NULL array", what);
        return false;
    }
    const void *arrs[] = {warped_rgba, warped_depth, alpha, fused_depth};
    for (const void *q : arrs)
        if (!aligned(q, 16)) {
            *st = fail(GVS_ERR_INVALID_ARG, "%s: arrays must be 16-byte aligned", what);
            return false;
        }
    return true;
}

gvs::BlendArgs blend_args(int32_t n_views, int32_t Wt, int32_t Ht, const uint32_t *warped_rgba,
                          const float *warped_depth, const uint8_t *alpha, const float *fused_depth) {
    gvs::BlendArgs a;
    memset(&a, 0, sizeof(a));
    a.K = n_views;
    a.Wt = Wt;
    a.Ht = Ht;
    a.rgba = warped_rgba;
    a.wdepth = warped_depth;
    a.alpha = alpha;
    a.fused = fused_depth;
    return a;
}

}  // namespace

extern "C" {

gvs_status gvs_blend_features(const gvs_camera *in_cams, int32_t n_views, const gvs_camera *target,
                              const uint32_t *warped_rgba, const float *warped_depth, const uint8_t *alpha,
                              const float *fused_depth, int32_t out_dtype, void *features, void *stream) {
    const Range nvtx_range("gvs_blend_features");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "blend features: target camera invalid");
    if (!in_cams) return fail(GVS_ERR_INVALID_ARG, "blend features: in_cams is NULL");
    gvs_status st = GVS_OK;
    if (!blend_common(n_views, target->width, target->height, warped_rgba, warped_depth, alpha, fused_depth,
                      "blend features", &st))
        return st;
    for (int k = 0; k < n_views; ++k)
        if (!camera_ok(&in_cams[k])) return fail(GVS_ERR_INVALID_ARG, "blend features: camera %d invalid", k);
    if (out_dtype != GVS_F32 && out_dtype != GVS_F16 && out_dtype != GVS_BF16)
        return fail(GVS_ERR_UNSUPPORTED, "blend features: out_dtype must be GVS_F32, GVS_F16 or GVS_BF16");
    if (!features || !aligned(features, 16)) return fail(GVS_ERR_INVALID_ARG, "blend features: features NULL or unaligned");
    gvs::BlendArgs a = blend_args(n_views, target->width, target->height, warped_rgba, warped_depth, alpha, fused_depth);
    a.fx = (float)target->fx;
    a.fy = (float)target->fy;
    a.cx = (float)target->cx;
    a.cy = (float)target->cy;
    // centres and axes in FP64, rounded once
    double ct[3];
    for (int r = 0; r < 3; ++r)
        ct[r] = -(target->R[0 + r] * target->t[0] + target->R[3 + r] * target->t[1] + target->R[6 + r] * target->t[2]);
    for (int k = 0; k < n_views; ++k) {
        const gvs_camera &c = in_cams[k];
        double cw[3], s = 0.0, ax = 0.0;
        for (int r = 0; r < 3; ++r) cw[r] = -(c.R[0 + r] * c.t[0] + c.R[3 + r] * c.t[1] + c.R[6 + r] * c.t[2]);
        for (int r = 0; r < 3; ++r) {
            a.ck[k][r] = (float)(target->R[3 * r + 0] * cw[0] + target->R[3 * r + 1] * cw[1] +
                                 target->R[3 * r + 2] * cw[2] + target->t[r]);
            s += (cw[r] - ct[r]) * (cw[r] - ct[r]);
            ax += c.R[6 + r] * target->R[6 + r];
        }
        a.dist[k] = (float)sqrt(s);
        a.axis[k] = (float)ax;
    }
    cudaError_t e = gvs::launch_blend_features(a, out_dtype, features, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend features: launch");
    return GVS_OK;
}

size_t gvs_blend_workspace_bytes(int32_t target_width, int32_t target_height) {
    if (target_width < 1 || target_height < 1) return 0;
    return align_up((size_t)gvs::blend_blocks(target_width, target_height) * sizeof(double), 256);
}

gvs_status gvs_blend(int32_t n_views, int32_t target_width, int32_t target_height, const uint32_t *warped_rgba,
                     const uint8_t *alpha, const float *warped_depth, const float *fused_depth, int32_t weight_dtype,
                     const void *w, const void *w_bg, const void *i_bg, float *image, double *l_depth,
                     void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_blend");
    gvs_status st = GVS_OK;
    if (!blend_common(n_views, target_width, target_height, warped_rgba, warped_depth, alpha, fused_depth, "blend",
                      &st))
        return st;
    if (weight_dtype != GVS_F32 && weight_dtype != GVS_BF16)
        return fail(GVS_ERR_UNSUPPORTED, "blend: weight_dtype must be GVS_F32 or GVS_BF16");
    if (!w || !w_bg || !i_bg || !image) return fail(GVS_ERR_INVALID_ARG, "blend: NULL array");
    const void *arrs[] = {image, l_depth};
    for (const void *q : arrs)
        if (q && !aligned(q, 8)) return fail(GVS_ERR_INVALID_ARG, "blend: outputs must be 8-byte aligned");
    const size_t need = gvs_blend_workspace_bytes(target_width, target_height);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
        return fail(GVS_ERR_WORKSPACE, "blend: workspace needs at least %zu bytes, 256-byte aligned", need);
    gvs::BlendArgs a = blend_args(n_views, target_width, target_height, warped_rgba, warped_depth, alpha, fused_depth);
    cudaError_t e = gvs::launch_blend(a, weight_dtype, w, w_bg, i_bg, image, l_depth,
                                      reinterpret_cast<double *>(workspace), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "blend: launch");
    return GVS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sphere-tracing raymarch (Supplement A.1).
// ---------------------------------------------------------------------------
extern "C" {

gvs_status gvs_fuse_depth_sphere(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                                 const gvs_camera *target, const gvs_sphere_params *params, float *fused_depth,
                                 int32_t *evals, void *workspace, size_t workspace_bytes, void *stream) {
    const Range nvtx_range("gvs_fuse_depth_sphere");
    int32_t W = 0, H = 0;
    if (!params) return fail(GVS_ERR_INVALID_ARG, "sphere: params is NULL");
    if (!views_ok(in_cams, n_views, &W, &H))
        return fail(GVS_ERR_INVALID_ARG, "sphere: input cameras invalid, of different sizes, or n_views out of range");
    if (!camera_ok(target)) return fail(GVS_ERR_INVALID_ARG, "sphere: target camera invalid");
    const gvs_sphere_params &p = *params;
    if (!(isfinite(p.z_near) && isfinite(p.z_far) && p.z_near > 0.0f && p.z_near < p.z_far))
        return fail(GVS_ERR_INVALID_ARG, "sphere: need 0 < z_near < z_far");
    gvs_status s = check_weight_params(p.mu, p.weight_const, p.window);
    if (s != GVS_OK) return s;
    if (p.max_steps < 1 || p.max_steps > (1 << 20)) return fail(GVS_ERR_INVALID_ARG, "sphere: max_steps in [1, 2^20]");
    if (!(isfinite(p.min_frac) && p.min_frac > 0.0f && p.min_frac <= 1.0f))
        return fail(GVS_ERR_INVALID_ARG, "sphere: min_frac must be in (0, 1]");
    if (p.depth_dtype != GVS_F32 && p.depth_dtype != GVS_F16)
        return fail(GVS_ERR_UNSUPPORTED, "sphere: depth_dtype must be GVS_F32 or GVS_F16");
    if (!fused_depth || !aligned(fused_depth, 16) || (evals && !aligned(evals, 16)))
        return fail(GVS_ERR_INVALID_ARG, "sphere: outputs NULL or not 16-byte aligned");
    if (n_views > 0 && (!in_depths || !aligned(in_depths, 16)))
        return fail(GVS_ERR_INVALID_ARG, "sphere: in_depths is NULL or misaligned");
    const size_t need = gvs_fuse_workspace_bytes(n_views, W, H);
    if (n_views > 0 && (!workspace || workspace_bytes < need || !aligned(workspace, 256)))
        return fail(GVS_ERR_WORKSPACE, "sphere: workspace needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = (cudaStream_t)stream;
    if (n_views > 0) {
        cudaError_t e = gvs::launch_weight_map(in_depths, p.depth_dtype, workspace, GVS_F32, n_views, W, H, p.mu,
                                               p.weight_const, p.window, st, true);
        if (e != cudaSuccess) return cuda_fail(e, "sphere: weight map launch");
    }
    gvs_fuse_params fp;
    memset(&fp, 0, sizeof(fp));
    fp.num_samples = 2;
    fp.z_near = p.z_near;
    fp.z_far = p.z_far;
    fp.mu = p.mu;
    fp.map_dtype = GVS_F32;
    gvs::SphereArgs a;
    memset(&a, 0, sizeof(a));
    a.f = fuse_args(in_cams, workspace, n_views, W, H, target, fp, fused_depth, nullptr);
    a.zf = p.z_far;
    a.c08mu = (float)(0.8 * (double)p.mu);
    a.min_frac = p.min_frac;
    a.max_steps = p.max_steps;
    a.evals = evals;
    cudaError_t e = gvs::launch_sphere(a, st);
    if (e != cudaSuccess) return cuda_fail(e, "sphere: launch");
    return GVS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Debug builds: the first out-of-range gather / scatter index.
// ---------------------------------------------------------------------------
extern "C" {

uint32_t gvs_take_device_status(void) { return gvs::async_timeouts_take(); }

uint64_t gvs_debug_bounds_error(void) {
    const unsigned long long r[] = {gvs::bounds_take_fuse(),   gvs::bounds_take_fuse_batch(),
                                    gvs::bounds_take_fuse_bwd(), gvs::bounds_take_sphere(),
                                    gvs::bounds_take_splat(),  gvs::bounds_take_gauss()};
    for (unsigned long long v : r)
        if (v) return v;
    return 0;
}

}  // extern "C"
