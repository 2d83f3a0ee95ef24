/*
 * gvs.h -- C ABI of libgvs.so, the GB300 (sm_103a) geometry core of
 * "Geometry-guided Online 3D Video Synthesis with Multi-View Temporal
 * Consistency" (arXiv 2505.18932).
 *
 * The calls follow the paper's problem statement (Sec. 3, "Method"): fixed
 * calibrated cameras (intrinsics K, world->camera R, t), one RGB-D frame per
 * input view, a target camera; out come the target-view fused depth (Eq. 3,
 * Supplement A.1) and the per-view forward-rendered colour, depth and
 * coverage (Sec. 3.1, Supplement A.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory   : every array argument is a DEVICE pointer to caller-owned,
 *            densely packed memory (no row padding).  The library never
 *            allocates; scratch lives in a caller-provided workspace whose
 *            size the matching *_workspace_bytes() call returns.  Arrays
 *            must be 16-byte aligned; workspaces 256-byte aligned.
 * Layouts  : per-view arrays are [n_views][height][width], row-major.
 *            Colour is RGBA8 packed in one little-endian uint32 per pixel
 *            (R in the low byte); alpha is carried but never read.
 *            Depth is z-depth in metres, float32; a value <= 0 or not finite
 *            marks an invalid pixel.
 * Cameras  : host memory, read during the call only.  x_cam = R x_world + t,
 *            R row-major; pixel (i, j) has its centre at integer coordinates
 *            (column i, row j).  All input views of one call share one size.
 * Streams  : `stream` is a cudaStream_t (NULL = legacy default stream).
 *            Every call only enqueues work; outputs are ready once the stream
 *            reaches that point.  Calls that share a workspace must not run
 *            concurrently.
 * Errors   : arguments are checked on the host before anything is enqueued;
 *            on GVS_ERR_INVALID_ARG nothing is written.  A failed launch
 *            returns GVS_ERR_CUDA.  gvs_last_error() gives a message for the
 *            calling thread's last failure.  No C++ exception crosses the ABI.
 *
 * Address contracts (what makes integer maps reproducible bit for bit)
 * -------------------------------------------------------------------
 * For an ordered camera pair (to, from) the host composes in FP64, in this
 * order, and rounds each entry once to FP32:
 *   Q = R_to R_from^T  (Q[r][c] = sum_m R_to[r][m] R_from[c][m], m = 0,1,2)
 *   g = t_to - Q t_from
 *   N = K_to Q,  b = K_to g   (row 0: fx*row0 + cx*row2; row 1: fy*row1 + cy*row2)
 *   M[r][0] = N[r][0]/fx_from,  M[r][1] = N[r][1]/fy_from,
 *   M[r][2] = (N[r][2] - N[r][0]*cx_from/fx_from) - N[r][1]*cy_from/fy_from
 * so that depth * (M [i j 1]^T) + b are the homogeneous pixel coordinates in
 * `to` of pixel (i, j) of `from` at that depth.  All device arithmetic that
 * decides an integer uses correctly rounded FP32 operations in a fixed order
 * (given with each call below).
 */
#ifndef GVS_H_
#define GVS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GVS_API __attribute__((visibility("default")))
#else
#define GVS_API
#endif

#define GVS_MAX_VIEWS 32        /* input views per call */
#define GVS_MAX_DIM 16384       /* width and height limit of every image */
#define GVS_MAX_SAMPLES 32767   /* samples per ray (crossing index is int16) */
#define GVS_MAX_WINDOW 15       /* confidence window side (odd) */
#define GVS_MAX_BATCH_ITEMS 1024 /* (frame, target) items of one batched fusion */

typedef enum {
    GVS_OK = 0,
    GVS_ERR_INVALID_ARG = 1,   /* bad pointer, size, parameter or camera; nothing enqueued */
    GVS_ERR_UNSUPPORTED = 2,   /* valid request outside what this build implements */
    GVS_ERR_WORKSPACE = 3,     /* workspace missing, misaligned or too small */
    GVS_ERR_CUDA = 4,          /* a CUDA launch or runtime call failed */
    GVS_ERR_DEVICE = 5         /* no usable CUDA device */
} gvs_status;

/* Storage type of depth inputs and of the fusion map.  Arithmetic is FP32
 * whatever the storage: FP16 halves the bytes moved and gathered. */
typedef enum {
    GVS_F32 = 0,               /* float */
    GVS_F16 = 1,               /* IEEE half */
    GVS_BF16 = 2,              /* bfloat16 (colour of the soft splat only) */
    GVS_U8 = 3                 /* uint8 (binary difference masks) */
} gvs_dtype;

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;     /* pinhole intrinsics, pixels */
    double R[9];               /* world->camera rotation, row-major */
    double t[3];               /* world->camera translation */
} gvs_camera;

/* Temporal refinement (Sec. 3.2, Eq. 1-2), binary mask form. */
typedef struct {
    float tau;                 /* colour threshold in [0,1]; integer T = floor(255 * tau) */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16: element type of depth_t and depth_state */
} gvs_refine_params;

/* Temporal refinement, the paper's soft mask (Sec. 3.2, Eq. 1-2 as printed). */
typedef struct {
    float beta;                /* 0.6 in the paper: the mask's floor */
    float lambda_t;            /* 0.7 in the paper: colour-difference scale */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16 */
} gvs_refine_soft_params;

/* TSDF fusion (Supplement A.1, Eq. 3). */
typedef struct {
    int32_t num_samples;       /* D >= 2 uniform samples of target z-depth in [z_near, z_far] */
    float z_near, z_far;       /* 0 < z_near < z_far */
    float mu;                  /* truncation (metres) > 0; also clamps the weight's variation */
    float weight_const;        /* 0.001 in the paper */
    int32_t window;            /* w, odd, 1..GVS_MAX_WINDOW; 7 in the paper */
    int32_t normalize;         /* 0: S = sum w*clamp (paper); 1: S / W */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16: element type of in_depths */
    int32_t map_dtype;         /* GVS_F32: (d, omega) as float2; GVS_F16: as half2 (omega rounded to half) */
    int32_t variant;           /* 0..6: mapping, bundle shape, slab-test lengths and samples evaluated at
                                  once by the march (lane per ray: 0: 8x4, 1: 8x4 longer segments, 2: 16x2,
                                  3: 4x8, 4: 4x8 and 5: 8x4 with two samples at once, for 5..16 views;
                                  warp per ray: 6, its lanes over views x consecutive samples, for 5..32
                                  views); other view counts run variant 0.  Every variant gives the same
                                  result, the autotuner picks the fastest (0 = default) */
} gvs_fuse_params;

/* Forward splat (Sec. 3.1, Supplement A.3). */
typedef struct {
    int32_t footprint;         /* 1: pixel-sized footprint; 0: single nearest pixel */
    float max_half_width;      /* footprint half-width cap in target pixels (>= 0.5), e.g. 2 */
    float mu_guide;            /* guided mask: |warped depth - fused depth| <= mu_guide */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16: element type of in_depths */
    int32_t guide_reject;      /* 1: before the depth test, drop every candidate lying in front of the
                                  fused surface, h.z < fused_depth - mu_guide (FP32 subtraction), so the
                                  z-buffer keeps the nearest surface consistent with the fused depth
                                  (the alternative reading of the fused-depth guidance, Sec. 3.1);
                                  needs fused_depth; a fused depth of 0 (no crossing) drops nothing */
} gvs_splat_params;

/* Differentiable colour splat (Sec. 3.1 / Supplement A.3, pixel-sized Gaussians as weights). */
typedef struct {
    float max_half_width;      /* footprint half-width cap (>= 0.5), as gvs_splat_params */
    float mu_band;             /* front band: sources with z <= z_winner + mu_band are blended */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16 */
    int32_t color_dtype;       /* GVS_F32 (float RGBA) or GVS_BF16 (bfloat16 RGBA) */
} gvs_soft_splat_params;

/* Sphere-tracing raymarch of the image-based TSDF (Supplement A.1). */
typedef struct {
    float z_near, z_far;       /* march from z_near; stop past z_far (target z-depth, metres) */
    float mu;                  /* truncation (tau of the paper), metres */
    float weight_const;        /* 0.001 in the paper */
    int32_t window;            /* odd, 7 in the paper */
    int32_t max_steps;         /* march samples per ray at most (bisection samples not counted), 1..2^20 */
    float min_frac;            /* smallest step, as a fraction of 0.8 mu (0, 1], e.g. 1/16 */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16 */
} gvs_sphere_params;

/* Pixel-sized Gaussian forward render (Sec. 3.1, Supplement A.3). */
#define GVS_MAX_GAUSS_RADIUS 32
typedef struct {
    float scale_px;            /* world standard deviation of each Gaussian = scale_px * depth / fx of its
                                  source view, i.e. scale_px source pixels (0.5: one pixel wide at +-1 sigma) */
    int32_t max_radius;        /* cap on the screen-space radius in target pixels, 1..GVS_MAX_GAUSS_RADIUS */
    int32_t depth_dtype;       /* GVS_F32 or GVS_F16 */
} gvs_gauss_params;

/* Library identification and diagnostics. */
GVS_API const char *gvs_version(void);
GVS_API const char *gvs_status_string(gvs_status s);
/* Message of the calling thread's most recent failed call ("" if none). */
GVS_API const char *gvs_last_error(void);

/*
 * gvs_refine_depth -- temporal depth refinement, Sec. 3.2, Eq. 1 and Eq. 2,
 * with the difference mask taken as a hard decision:
 *   m(p)        = [ max_{c in R,G,B} |rgba_t_c(p) - rgba_prev_c(p)| > T ],
 *                 T = floor(255 * tau) (integers; alpha ignored)
 *   depth_state = m ? depth_t : depth_state       (in place, bit-exact copy)
 * rgba_prev == NULL marks the first frame: m = 1 everywhere.
 *   rgba_t, rgba_prev : uint32 [n_views][height][width]
 *   depth_t           : [n_views][height][width] of params->depth_dtype
 *   depth_state       : same type and shape, in: previous filtered
 *                       depth (ignored when rgba_prev == NULL), out: new one
 *   mask              : uint8  [n_views][height][width] or NULL
 */
GVS_API gvs_status gvs_refine_depth(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t,
                            void *depth_state, uint8_t *mask, int32_t n_views, int32_t width,
                            int32_t height, const gvs_refine_params *params, void *stream);

/* Workspace bytes for gvs_refine_depth_soft: two quarter-resolution float grids per view. */
GVS_API size_t gvs_refine_soft_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/*
 * gvs_refine_depth_soft -- temporal depth refinement with the soft difference
 * mask exactly as Sec. 3.2 prints it:
 *   M = min(|I^t - I^{t-1}| / lambda_t + beta, 1)               (Eq. 1)
 *   depth_state = M depth_t + (1 - M) depth_state               (Eq. 2)
 * with M computed at quarter resolution, 3x3 max-pooled and bilinearly
 * upsampled.  Readings: the per-pixel difference is the largest of the R, G,
 * B differences in [0, 1]; a quarter cell is the mean over its 4x4 pixels
 * (fewer at the right and bottom edges); pooling clamps at the borders; the
 * upsample samples the quarter grid at ((x + 0.5) / 4 - 0.5, (y + 0.5) / 4 -
 * 0.5), clamped to the grid.  Where the previous depth is invalid the new one
 * is taken; where the new one is invalid the previous one is kept.
 *   rgba_t, rgba_prev : uint32 [n_views][height][width] (both required)
 *   depth_t, depth_state : [n_views][height][width] of params->depth_dtype
 *   mask      : float [n_views][height][width] (M), or NULL
 *   workspace : >= gvs_refine_soft_workspace_bytes() bytes, 256-byte aligned
 */
GVS_API gvs_status gvs_refine_depth_soft(const uint32_t *rgba_t, const uint32_t *rgba_prev, const void *depth_t,
                                         void *depth_state, float *mask, int32_t n_views, int32_t width,
                                         int32_t height, const gvs_refine_soft_params *params, void *workspace,
                                         size_t workspace_bytes, void *stream);

/*
 * gvs_select_views -- the K input views closest to the target (Sec. 3.1; the
 * evaluation uses K = 4 or 2): ranked by the distance between camera centres
 * C = -R^T t, ties to the lower index.  Host only; writes k indices.
 */
GVS_API gvs_status gvs_select_views(const gvs_camera *cams, int32_t n, const gvs_camera *target, int32_t k,
                                    int32_t *out_idx);

/* Workspace bytes for gvs_fuse_depth (the "map" of gvs_weight_map): the packed
 * (depth, weight) float2 of every input pixel followed by per-view depth
 * bounds over 8, 32 and 128 pixel tiles and over the whole view. */
GVS_API size_t gvs_fuse_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/*
 * gvs_fuse_depth -- image-based TSDF fusion and zero-crossing extraction,
 * Supplement A.1 (projection, signed distance, confidence weight, omega = 0
 * behind the band) and Eq. 3 (raymarch), with D uniform samples.
 *
 * For target pixel (i, j) and sample s = 0..D-1 (FP32 contract):
 *   z_s = fma(s, dz, zn),  zn = (float)z_near,
 *         dz = (float)(((double)z_far - (double)z_near) / (D - 1))
 *   a   = M_k [i j 1]^T  by fma(M[r][0], i, fma(M[r][1], j, M[r][2]))
 *         with (M_k, b_k) composed for (to = view k, from = target)
 *   h   = fma(z_s, a, b_k);  the view contributes only if h.z > 1e-6
 *   (u, v) = nearest integers (ties to even) of the EXACT quotients
 *         h.x/h.z, h.y/h.z; the view contributes only if inside its image
 *   d   = depth_k(u, v); omega = confidence weight of view k at (u, v):
 *         nu = sum over the w x w window (clamped to the image) of
 *         min((d - d_n)^2, mu^2), an invalid neighbour counting mu^2;
 *         omega = min(weight_const * (nu / w^2)^(-1/2), 1), 1 if nu = 0,
 *         0 if d is invalid
 *   sdf = (d - h.z) / mu;  omega = 0 where sdf < -1 (hidden behind the band)
 *   S_s = sum_k omega_k clamp(sdf_k, -1, 1),  W_s = sum_k omega_k
 *         (normalize: S_s / W_s where W_s > 0)
 * fused_depth(i, j) = z_s + (z_{s+1} - z_s) S_s / (S_s - S_{s+1}) at the first
 *   s with W_s > 0, W_{s+1} > 0, S_s > 0, S_{s+1} <= 0; 0 if there is none.
 *   in_cams   : n_views cameras, all of one size (width x height)
 *   in_depths : [n_views][height][width] of params->depth_dtype (values are
 *               widened to FP32; with map_dtype GVS_F16 the weight is stored
 *               as half, every sum and the interpolation stay FP32)
 *   fused_depth : float [target.height][target.width]
 *   crossing  : int16 [target.height][target.width] (s, or -1) or NULL
 *   workspace : >= gvs_fuse_workspace_bytes(n_views, width, height) bytes
 */
GVS_API gvs_status gvs_fuse_depth(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                          const gvs_camera *target, const gvs_fuse_params *params, float *fused_depth,
                          int16_t *crossing, void *workspace, size_t workspace_bytes, void *stream);

/*
 * gvs_weight_map -- the two stages of gvs_fuse_depth, callable separately.
 * Stage 1: the confidence weight of Supplement A.1 at every input pixel.
 * With nearest-pixel sampling the weight at a sample is a function of the
 * sampled pixel only, so it is computed once per pixel and stored with the
 * depth as (d, omega), (0, 0) where d is invalid; with it go the min and max
 * valid depth of every 8, 32 and 128 pixel tile and of each whole view,
 * which let the march skip runs of samples that provably hold no crossing.
 *   in_depths : [n_views][height][width] of depth_dtype (GVS_F32 or GVS_F16)
 *   map_dtype : GVS_F32 or GVS_F16 storage of (d, omega); the map must be read
 *               back with the same map_dtype in gvs_fuse_params
 *   map       : >= gvs_fuse_workspace_bytes(n_views, width, height) bytes,
 *               256-byte aligned; its layout is private to the library
 */
GVS_API gvs_status gvs_weight_map(const void *in_depths, int32_t depth_dtype, int32_t n_views, int32_t width,
                                  int32_t height, float mu, float weight_const, int32_t window, int32_t map_dtype,
                                  void *map, size_t map_bytes, void *stream);

/*
 * gvs_fuse_depth_from_map -- stage 2: the TSDF march and zero crossing of
 * gvs_fuse_depth (Supplement A.1, Eq. 3) reading a map written by
 * gvs_weight_map for the same depths.  params->weight_const and
 * params->window are not used.
 */
GVS_API gvs_status gvs_fuse_depth_from_map(const gvs_camera *in_cams, const void *map, size_t map_bytes,
                                           int32_t n_views, const gvs_camera *target,
                                           const gvs_fuse_params *params, float *fused_depth, int16_t *crossing,
                                           void *stream);

/* Workspace bytes for gvs_fuse_depth_backward: one float2 accumulator per input pixel. */
GVS_API size_t gvs_fuse_backward_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/*
 * gvs_fuse_depth_backward -- adjoint of gvs_fuse_depth (normalize = 0):
 * grad_depths = d(sum_p grad_fused(p) D(p)) / d in_depths, written (not
 * accumulated).  D = z_s + dz S_s / (S_s - S_{s+1}) (Eq. 3 with linear
 * interpolation) is differentiated through S_s and S_{s+1} only, each
 * S = sum_k omega_k clamp(sdf_k, -1, 1) (Supplement A.1) through the clamped
 * signed distance (slope 1/mu strictly inside the band) and through the
 * confidence weight (d omega / d nu = -omega / (2 nu) unless saturated, nu
 * through every (d_c - d_n)^2 strictly below mu^2).  The nearest-pixel
 * choice, the cut-off, the crossing index and saturation are piecewise
 * constant and carry no gradient.  The two bracketing samples are recomputed;
 * nothing of size D x H x W is stored.
 *   in_depths, params : as passed to the forward (params->normalize must be 0)
 *   map       : the forward's map (gvs_weight_map / gvs_fuse_depth workspace)
 *   crossing  : the forward's int16 crossing index [Ht][Wt]
 *   grad_fused: float [Ht][Wt];  grad_depths: float [n_views][height][width]
 *   workspace : >= gvs_fuse_backward_workspace_bytes() bytes, 256-byte aligned
 * Gradient sums use float atomics: the order, hence the last bits, can vary
 * from run to run.
 */
GVS_API gvs_status gvs_fuse_depth_backward(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                                           const gvs_camera *target, const gvs_fuse_params *params,
                                           const void *map, size_t map_bytes, const int16_t *crossing,
                                           const float *grad_fused, float *grad_depths, void *workspace,
                                           size_t workspace_bytes, void *stream);

/* Workspace bytes for gvs_soft_splat: a 64-bit key and a float4 accumulator per
 * target pixel (one view at a time; a larger workspace holds several views). */
GVS_API size_t gvs_soft_splat_workspace_bytes(int32_t n_views, int32_t target_width, int32_t target_height);

/*
 * gvs_soft_splat -- differentiable forward rendering of each input view's
 * colour into the target (Sec. 3.1, Supplement A.3: pixel-sized Gaussians,
 * each view rendered separately, occlusion by depth).  The winner, warped depth
 * and alpha are exactly those of gvs_forward_splat in footprint mode (same
 * contract).  The colour blends every covering source q within the front band
 * z_q <= z_winner + mu_band (FP32 sum and test) with weights
 *   g_q = exp(-|(x_q, y_q) - p|^2 / (2 sigma_q^2)),  sigma_q = hw_q / 2:
 *   colour(p) = sum g_q c_q / sum g_q   (RGB; the 4th channel is written 0).
 *   in_color    : [n_views][height][width][4] of color_dtype, values in [0, 1]
 *   winner      : int32 [n_views][Ht][Wt];  warped_color: float [n_views][Ht][Wt][4]
 *   warped_depth: float [n_views][Ht][Wt] (NULL allowed); alpha: uint8 (NULL allowed)
 *   weight_sum  : float [n_views][Ht][Wt], sum g (kept for the backward)
 */
GVS_API gvs_status gvs_soft_splat(const gvs_camera *in_cams, const void *in_depths, const void *in_color,
                                  int32_t n_views, const gvs_camera *target, const gvs_soft_splat_params *params,
                                  int32_t *winner, float *warped_color, float *warped_depth, float *weight_sum,
                                  uint8_t *alpha, void *workspace, size_t workspace_bytes, void *stream);

/*
 * gvs_soft_splat_backward -- adjoint of gvs_soft_splat (Sec. 3.1 and Supplement
 * A.3, differentiated with respect to the source depths and colours).  From the upstream
 * gradients of the warped colour (grad_color [n_views][Ht][Wt][4], 4th channel
 * ignored) and, optionally, of the warped depth (grad_depth [n_views][Ht][Wt]),
 * writes the gradients of the source depths (grad_in_depth float [n_views][H][W])
 * and colours (grad_in_color float [n_views][H][W][4], 4th channel 0):
 *   d colour / d c_q = g_q / sum g,   d colour / d g_q = (c_q - colour) / sum g,
 *   g_q through (x_q, y_q) and sigma_q as functions of d_q (sigma only where the
 *   half-width is not clamped), and the warped depth through dz/dd of the
 *   winner.  Band membership, coverage and the winner are piecewise constant.
 * Needs the forward's winner, warped_color, warped_depth and weight_sum.  One
 * thread per source pixel gathers over its own footprint: no atomics, so the
 * result is deterministic.
 */
GVS_API gvs_status gvs_soft_splat_backward(const gvs_camera *in_cams, const void *in_depths, const void *in_color,
                                           int32_t n_views, const gvs_camera *target,
                                           const gvs_soft_splat_params *params, const int32_t *winner,
                                           const float *warped_color, const float *warped_depth,
                                           const float *weight_sum, const float *grad_color, const float *grad_depth,
                                           float *grad_in_depth, float *grad_in_color, void *stream);

/*
 * Batched fusion: many (frame, target) items in one persistent launch (a serving
 * pattern; the paper has no counterpart, each item is Supplement A.1's fusion).  Each
 * item fuses the map of one frame (gvs_weight_map) into one target camera,
 * exactly as gvs_fuse_depth_from_map would; targets may differ in size.  The
 * launch keeps every SM busy with one grid that takes bundles of target pixels
 * from a global counter until all items are done (no block waits on another),
 * and is a plain kernel launch plus a 4-byte reset, so it can be captured in a
 * CUDA graph.
 */
typedef struct {
    const void *map;           /* the frame's map, as from gvs_weight_map */
    size_t map_bytes;
    const gvs_camera *target;  /* host, read during gvs_fuse_batch_create */
    float *fused_depth;        /* device [target.height][target.width] */
    int16_t *crossing;         /* device, or NULL */
} gvs_fuse_item;

typedef struct gvs_fuse_batch gvs_fuse_batch;  /* opaque host object */

/* Device table bytes for n_items items. */
GVS_API size_t gvs_fuse_batch_bytes(int32_t n_items);

/* Validates the items (all with the same input views and params), writes their
 * descriptors into `table` (device, caller-owned, >= gvs_fuse_batch_bytes)
 * with a synchronous copy -- call it outside any stream capture -- and returns
 * a host handle.  The maps, outputs and table must outlive the handle. */
GVS_API gvs_status gvs_fuse_batch_create(const gvs_camera *in_cams, int32_t n_views, const gvs_fuse_item *items,
                                         int32_t n_items, const gvs_fuse_params *params, void *table,
                                         size_t table_bytes, gvs_fuse_batch **out);

/* Enqueues the batched fusion on `stream`.  Launches that share a table must
 * not overlap. */
GVS_API gvs_status gvs_fuse_batch_launch(const gvs_fuse_batch *batch, void *stream);

GVS_API void gvs_fuse_batch_destroy(gvs_fuse_batch *batch);

/*
 * The temporal term of Sec. 3.2 / Supplement A.2, for a novel viewpoint that
 * stays fixed from frame to frame (or whose state the caller reprojects):
 *
 * gvs_temporal_weight -- the target-view difference mask M(p) = max over views
 * of each view's mask at its z-buffer winner (the forward splat of the masks
 * with a channel-wise maximum; 1 where no view covers p), and the temporal
 * fusion weight
 *   w_tmp(p) = min(beta_t (w_tmp_prev(p) + w_view_prev(p)) max(1 - M(p), 0), eta)
 * where w_view_prev is the views' weight at the previous frame's crossing
 * (view_weight of gvs_fuse_depth_temporal).  eta = 15 in the paper; beta_t is
 * not given there (1 is this library's default).
 *   masks       : [n_views][height][width], float (soft masks) or uint8 (binary)
 *   winner      : int32 [n_views][target_height][target_width] (gvs_forward_splat)
 *   w_tmp_prev, w_view_prev, w_tmp, target_mask (or NULL): float [Ht][Wt]
 */
GVS_API gvs_status gvs_temporal_weight(const void *masks, int32_t mask_dtype, const int32_t *winner,
                                       int32_t n_views, int32_t width, int32_t height, int32_t target_width,
                                       int32_t target_height, const float *w_tmp_prev, const float *w_view_prev,
                                       float beta_t, float eta, float *w_tmp, float *target_mask, void *stream);

/*
 * gvs_fuse_depth_temporal -- Supplement A.2: gvs_fuse_depth_from_map with the previous output
 * depth prev_depth(p) as one more TSDF input at the ray's own pixel, weighted
 * w_tmp(p) (zero or an invalid depth: absent):
 *   S_s += w_tmp clamp((prev_depth - z_s) / mu, -1, 1), W_s += w_tmp,
 * both only where (prev_depth - z_s) / mu >= -1, as for the views.
 *   view_weight : float [Ht][Wt] (or NULL): the views' weight sum at the
 *                 crossing, interpolated like the depth (0 without a crossing)
 */
GVS_API gvs_status gvs_fuse_depth_temporal(const gvs_camera *in_cams, const void *map, size_t map_bytes,
                                           int32_t n_views, const gvs_camera *target, const gvs_fuse_params *params,
                                           const float *prev_depth, const float *w_tmp, float *fused_depth,
                                           int16_t *crossing, float *view_weight, void *stream);

/* gvs_guided_mask -- the guided mask of gvs_forward_splat (the fused depth guiding
 * the warped views, Sec. 3.1 and Sec. 3.3) computed afterwards:
 * guided = alpha && |warped_depth - fused_depth| <= mu_guide, all [n_views][Ht][Wt]
 * except fused_depth [Ht][Wt]. */
GVS_API gvs_status gvs_guided_mask(const float *warped_depth, const uint8_t *alpha, const float *fused_depth,
                                   int32_t n_views, int32_t target_width, int32_t target_height, float mu_guide,
                                   uint8_t *guided, void *stream);

/* Workspace bytes for gvs_forward_splat: one 64-bit z-buffer of the target size.
 * A workspace holding several such buffers lets several views splat in one pass. */
GVS_API size_t gvs_splat_workspace_bytes(int32_t n_views, int32_t target_width, int32_t target_height);

/*
 * gvs_forward_splat -- per-view forward rendering into the target camera with
 * a depth test, Sec. 3.1 and Supplement A.3 (each view rendered separately,
 * fully opaque pixel-sized primitives, occlusion by depth).
 *
 * For source pixel (u, v) of view k with valid depth d (FP32 contract, with
 * (A, c) composed for (to = target, from = view k), f = fx_target / fx_k):
 *   m = A [u v 1]^T by fma as above;  h = fma(d, m, c);  skip unless h.z > 1e-6
 *   x = h.x / h.z,  y = h.y / h.z            (correctly rounded FP32)
 *   footprint: rho = f * (d / h.z);  hw = min(max(0.5 * rho, 0.5), max_half_width)
 *              covers target pixels ceil(x - hw)..floor(x + hw) (and y alike)
 *   point    : covers (rint(x), rint(y))
 *   key = (float bits of h.z) << 32 | (v * width + u); per target pixel the
 *   smallest key wins: the nearest surface, ties to the lower source index.
 *   guide_reject: a candidate for target pixel p with h.z < fused_depth[p] - mu_guide
 *   takes no part in the depth test at p.
 * in_depths is [n_views][height][width] of params->depth_dtype (widened to FP32).
 * Outputs, each [n_views][target.height][target.width] (NULL to skip, except winner):
 *   winner       int32  source pixel index v*width+u, or -1
 *   warped_rgba  uint32 source colour of the winner (0 if none)
 *   warped_depth float  h.z of the winner (0 if none)
 *   alpha        uint8  1 where a winner exists
 *   guided       uint8  alpha && |warped_depth - fused_depth| <= mu_guide;
 *                needs fused_depth [target.height][target.width]
 *   workspace : >= gvs_splat_workspace_bytes(...) bytes
 */
GVS_API gvs_status gvs_forward_splat(const gvs_camera *in_cams, const void *in_depths, const uint32_t *in_rgba,
                             int32_t n_views, const gvs_camera *target, const gvs_splat_params *params,
                             const float *fused_depth, int32_t *winner, uint32_t *warped_rgba,
                             float *warped_depth, uint8_t *alpha, uint8_t *guided, void *workspace,
                             size_t workspace_bytes, void *stream);

/*
 * gvs_forward_splat_noalloc -- gvs_forward_splat for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a service of
 * the library.  A plugin living inside a host application that owns all device
 * allocations, code recorded into a CUDA graph, or a real-time loop that must
 * not block on the allocator cannot create the splat workspace; this call
 * needs none.  Its z-buffer is a file-scope device array of 2^21 64-bit keys
 * (16 MiB) that every GPU loading the library holds until the process exits.
 *   - Arguments, outputs and errors are those of gvs_forward_splat without the
 *     workspace.  Targets of more than 2,097,152 pixels (e.g. larger than
 *     1920 x 1080) are rejected with GVS_ERR_INVALID_ARG before anything runs.
 *   - The array exists once per CUDA context that loads the library (the
 *     device's primary context, a context the caller created, the primary
 *     context created again after cudaDeviceReset).  The first call in a
 *     context looks up that context's copy with cudaGetSymbolAddress (with the
 *     context current) and caches it under the driver's unique context id;
 *     make that first call before any stream capture.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - Every call shares the one array and clears it before use.  Calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on it:
 *     order them on one stream.
 */
GVS_API gvs_status gvs_forward_splat_noalloc(const gvs_camera *in_cams, const void *in_depths,
                                             const uint32_t *in_rgba, int32_t n_views, const gvs_camera *target,
                                             const gvs_splat_params *params, const float *fused_depth,
                                             int32_t *winner, uint32_t *warped_rgba, float *warped_depth,
                                             uint8_t *alpha, uint8_t *guided, void *stream);

/*
 * gvs_gauss_splat -- Sec. 3.1 and Supplement A.3 as the paper renders them: every
 * input pixel becomes an isotropic, fully opaque 3D Gaussian (colour = the pixel,
 * position from its depth, scale one source pixel) and each input view is rendered
 * separately into the target with the rasterisation rules of 3D Gaussian splatting
 * (Kerbl et al. 2023).  For source pixel (u, v) of view k with valid depth d:
 *   x, y, h.z, rho      the splat contract of gvs_forward_splat (footprint mode)
 *   a = (x - cx) / fx,  b = (y - cy) / fy,  q = fy / fx   (target intrinsics as FP32)
 *   Sigma = (scale_px rho)^2 [[1 + a^2, q a b], [q a b, q^2 (1 + b^2)]] + 0.3 I
 *           (the EWA projection of the isotropic Gaussian plus the 0.3 px^2 dilation)
 *   r = min(ceil(3 sqrt(mid + sqrt(max(0.1, mid^2 - det(Sigma))))), max_radius),
 *       mid = (Sigma_xx + Sigma_yy) / 2
 *   covered target pixels i in [ceil(x - r), floor(x + r)], j alike
 * All of the above in FP32, each operation rounded as written (no contraction).
 * Per target pixel (i, j) the covering Gaussians in ascending key
 * (float bits of h.z) << 32 | (v * width + u)   (nearest first, ties to the lower index):
 *   alpha = min(0.99, exp(-0.5 (dx, dy) Sigma^-1 (dx, dy)^T)), (dx, dy) = (x - i, y - j);
 *   alpha < 1/255: skipped;  T' = T (1 - alpha) < 1e-4: the walk stops before it;
 *   otherwise C += colour * alpha * T, Z += h.z * alpha * T, A += alpha * T, T = T'.
 * Outputs, [n_views][target.height][target.width]:
 *   color  float4 (C.r, C.g, C.b, 1 - T): colour premultiplied (black background), opacity
 *   depth  float  Z / A (0 where nothing lands)
 * Colours are the RGBA8 channels / 255 (alpha channel unused).  workspace: at least
 * gvs_gauss_splat_workspace_bytes(width, height, target width, target height, max_radius)
 * bytes, 256-byte aligned; it holds per-pixel records and per-16x16-tile key lists.
 */
GVS_API size_t gvs_gauss_splat_workspace_bytes(int32_t width, int32_t height, int32_t target_width,
                                               int32_t target_height, int32_t max_radius);
GVS_API gvs_status gvs_gauss_splat(const gvs_camera *in_cams, const void *in_depths, const uint32_t *in_rgba,
                                   int32_t n_views, const gvs_camera *target, const gvs_gauss_params *params,
                                   float *color, float *depth, void *workspace, size_t workspace_bytes,
                                   void *stream);

/*
 * gvs_fuse_depth_sphere -- Supplement A.1's own raymarch: from z_near advance along
 * each target ray by 0.8 s until s changes sign, then three bisection steps.
 * s is the fused signed distance of the uniform march (same projection, nearest
 * pixel, cut-off and clamp; gvs_fuse_depth), normalised: s_n = S / W.  Per ray, in
 * FP32 with every operation rounded as written:
 *   z = z_near;  while z <= z_far and fewer than max_steps samples:
 *     evaluate S, W at z;
 *     if the previous sample had W > 0, S > 0 and this one W > 0, S <= 0:
 *       lo, hi = previous z, z; three times: m = 0.5 (lo + hi), lo = m if W(m) > 0 and
 *       S(m) > 0 else hi = m;  depth = 0.5 (lo + hi); stop
 *     z = z + fl32(0.8 mu) * (W > 0 ? max(S / W, min_frac) : 1)
 *   no crossing: depth 0.
 * The confidence weights are computed with correctly rounded operations
 * (omega = min(weight_const / sqrt(nu / window^2), 1), nu summed in raster order by
 * fused multiply-adds), so the whole march is reproducible bit for bit.
 * fused_depth [target.height][target.width]; evals (NULL to skip) the samples
 * evaluated per ray, bisection samples included.  workspace:
 * gvs_fuse_workspace_bytes(n_views, width, height) (it receives the (d, omega) map).
 */
GVS_API gvs_status gvs_fuse_depth_sphere(const gvs_camera *in_cams, const void *in_depths, int32_t n_views,
                                         const gvs_camera *target, const gvs_sphere_params *params,
                                         float *fused_depth, int32_t *evals, void *workspace,
                                         size_t workspace_bytes, void *stream);

/*
 * gvs_blend_features -- the input of the blending network (Sec. 3.3; the
 * supplement's list of network inputs), (9K + 1) channel planes
 * [9K + 1][target.height][target.width] of out_dtype (GVS_F32, GVS_F16 or GVS_BF16), in order:
 *   3K  forward-rendered colours, view-major, channel byte / 255 (R, G, B of warped_rgba)
 *   K   their depths (warped_depth)            K   their alphas (0 or 1)
 *   1   the TSDF depth D (fused_depth)
 *   K   n . d_k    K   r_t . d_k    K   |c_k - c_t|    K   z_k . z_t
 * with P the target-camera point of pixel (i, j) at depth D, n the normal of D at
 * (i, j) from central differences of the back-projected points (formed as
 * ((delta (i - cx) + sigma) / fx, delta (j - cy) / fy, delta), delta = D(i+1) - D(i-1),
 * sigma = D(i+1) + D(i-1), and alike vertically), turned to face the camera and
 * normalised, 0 where (i, j) or a 4-neighbour has no depth or lies on the border;
 * d_k the unit vector from view k's centre to P; r_t = P / |P|; c the camera centres;
 * z the optical axes; all in the target frame.  n . d_k and r_t . d_k are 0 where D
 * is 0.  Inputs as gvs_forward_splat writes them, [n_views][target.height][target.width].
 */
GVS_API gvs_status gvs_blend_features(const gvs_camera *in_cams, int32_t n_views, const gvs_camera *target,
                                      const uint32_t *warped_rgba, const float *warped_depth,
                                      const uint8_t *alpha, const float *fused_depth, int32_t out_dtype,
                                      void *features, void *stream);

/*
 * gvs_blend -- Eq. 4 and Eq. 5 with L_Depth (Sec. 3.3):
 *   I_FG = sum_k I_k a_k w_k / sum_k a_k w_k   (0 where the sum is 0; the printed
 *          denominator is read as the sum over views)
 *   image = (1 - w_BG) I_FG + w_BG I_BG                         [3][Ht][Wt] float
 *   l_depth = 1/(Ht Wt K) sum_p | D(p) - sum_k D_k a_k w_k / sum_k a_k w_k |   (one double)
 * w [n_views][Ht][Wt], w_bg [Ht][Wt], i_bg [3][Ht][Wt] of weight_dtype (GVS_F32 or
 * GVS_BF16): the network's output planes.  l_depth may be NULL.  The reduction is
 * in a fixed order (bit-reproducible).  workspace: gvs_blend_workspace_bytes(...).
 */
GVS_API size_t gvs_blend_workspace_bytes(int32_t target_width, int32_t target_height);
GVS_API gvs_status gvs_blend(int32_t n_views, int32_t target_width, int32_t target_height,
                             const uint32_t *warped_rgba, const uint8_t *alpha, const float *warped_depth,
                             const float *fused_depth, int32_t weight_dtype, const void *w, const void *w_bg,
                             const void *i_bg, float *image, double *l_depth, void *workspace,
                             size_t workspace_bytes, void *stream);

/*
 * gvs_uniform_blend_loss -- the training loss of Sec. 3.3 (0.8 L1 + 0.1 L_Depth in
 * the paper) on the blend of the differentiable splat's views with uniform weights
 * (Eq. 4 with every w_k = 1, its denominator read as the sum over the views), and
 * its gradient.  Per target pixel p, with a_k the views' alpha (0/1):
 *   A = sum_k a_k,  B = sum_k a_k I_k / A   (I_k = warped_color RGB; n pixels have A > 0)
 *   L1 = sum_{A > 0} sum_rgb |B - GT| / (3 n)
 *   Dbar = sum_k a_k D_k / A,  v = [A > 0 and F > 0]   (D_k warped depth, F fused depth)
 *   L_Depth = sum_p v |F - Dbar| / (n_views Ht Wt)       (the printed 1/(HWK))
 *   L = w_l1 L1 + w_depth L_Depth
 * FP32 per pixel and over each GPU thread's and warp's pixels (non-negative terms: each
 * such sum within (terms + 5) 2^-24 of its value), FP64 beyond; every sum in an order
 * fixed by the target size alone (deterministic).
 *   warped_color : float [n_views][Ht][Wt][4] (4th channel unused), 16-byte aligned
 *   alpha        : uint8 [n_views][Ht][Wt];  warped_depth: float [n_views][Ht][Wt]
 *   fused_depth  : float [Ht][Wt];  ground_truth: float [Ht][Wt][3]
 *   loss         : device double[3] = {L, L1, L_Depth}
 *   grad_pixel   : float [Ht][Wt][4] or NULL: dL/dI_k (RGB) and dL/dD_k (4th) shared by
 *                  every view k with a_k = 1 at the pixel (0 at uncovered pixels):
 *                  w_l1 sign(B - GT) / (3 n A) and -w_depth v sign(F - Dbar) / (n_views Ht Wt A)
 *   grad_fused   : float [Ht][Wt] or NULL: dL/dF = w_depth v sign(F - Dbar) / (n_views Ht Wt)
 *                  (|x|' = sign(x), 0 at 0)
 *   workspace    : >= gvs_uniform_blend_loss_workspace_bytes(Wt, Ht), 256-byte aligned
 * Errors: GVS_ERR_INVALID_ARG for bad sizes, weights, NULL or misaligned arrays;
 * GVS_ERR_WORKSPACE for a short workspace.
 */
GVS_API size_t gvs_uniform_blend_loss_workspace_bytes(int32_t target_width, int32_t target_height);
GVS_API gvs_status gvs_uniform_blend_loss(int32_t n_views, int32_t target_width, int32_t target_height,
                                          const float *warped_color, const uint8_t *alpha,
                                          const float *warped_depth, const float *fused_depth,
                                          const float *ground_truth, float w_l1, float w_depth, double *loss,
                                          float *grad_pixel, float *grad_fused, void *workspace,
                                          size_t workspace_bytes, void *stream);

/*
 * gvs_uniform_blend_loss_grad -- the gradient of the loss that the last
 * gvs_uniform_blend_loss call on `workspace` computed (same target size; the
 * workspace keeps each pixel's blend signs and the two scales between the calls),
 * multiplied by the upstream gradient *grad_loss: what a backward pass needs when
 * the loss feeds further arithmetic, with the scalar read on the device (no host
 * round trip, and the call can be captured in a CUDA graph).
 *   grad_loss  : device float, or NULL for 1 (then the outputs equal those of
 *                gvs_uniform_blend_loss bit for bit); otherwise each output is the
 *                unit-upstream value times *grad_loss, rounded once
 *   grad_pixel : float [Ht][Wt][4] or NULL, 16-byte aligned; grad_fused: float [Ht][Wt] or NULL
 *                (as gvs_uniform_blend_loss defines them); at least one of the two
 *   workspace  : the one the loss call used, not written in between; only read here
 * Errors: GVS_ERR_INVALID_ARG for bad sizes, no output or misaligned arrays;
 * GVS_ERR_WORKSPACE for a short or misaligned workspace.  A workspace that no loss
 * call has filled gives undefined (finite or not) gradients, never an access outside it.
 */
GVS_API gvs_status gvs_uniform_blend_loss_grad(int32_t target_width, int32_t target_height, const float *grad_loss,
                                               float *grad_pixel, float *grad_fused, const void *workspace,
                                               size_t workspace_bytes, void *stream);

/*
 * gvs_soft_splat_backward_blended -- gvs_soft_splat_backward for a loss that sees the
 * views only through their uniform blend (as gvs_uniform_blend_loss): the upstream
 * gradients are one per target pixel, shared by every view that covers it,
 * grad_pixel float [Ht][Wt][4] = (dL/d colour RGB, dL/d warped depth), in place of
 * grad_color and grad_depth [n_views][Ht][Wt].  The result equals
 * gvs_soft_splat_backward given grad_color_k = a_k grad_pixel.rgb and grad_depth_k =
 * a_k grad_pixel.w, without those per-view arrays.  Other arguments, outputs and
 * errors as gvs_soft_splat_backward.
 */
GVS_API gvs_status gvs_soft_splat_backward_blended(const gvs_camera *in_cams, const void *in_depths,
                                                   const void *in_color, int32_t n_views, const gvs_camera *target,
                                                   const gvs_soft_splat_params *params, const int32_t *winner,
                                                   const float *warped_color, const float *warped_depth,
                                                   const float *weight_sum, const float *grad_pixel,
                                                   float *grad_in_depth, float *grad_in_color, void *stream);

/*
 * gvs_take_device_status -- a service of the library (the paper has no counterpart).
 * Kernels that stage their inputs in shared memory with asynchronous bulk copies
 * (the hard splat's resolve) wait for those copies a bounded time (about 2^24
 * polls of the completion barrier); a block whose wait gives up writes none of
 * its outputs and is counted here.  Returns the count since the last call (0 in
 * normal operation) and clears it; read it after the stream has synchronised.
 * Nothing traps and nothing waits without a limit.
 */
GVS_API uint32_t gvs_take_device_status(void);

/*
 * gvs_debug_bounds_error -- a service of the library (the paper has no counterpart).
 * In a build compiled with GVS_BOUNDS_CHECK every kernel checks its computed
 * gather / scatter indices (fusion map and bound tiles, splat keys and colour
 * gathers, Gaussian records and tile lists), skips an out-of-range access and records
 * the first one; this returns ((site << 48) | index) of that access, 0 if none, and
 * clears the record.  A normal build checks nothing and always returns 0.
 */
GVS_API uint64_t gvs_debug_bounds_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GVS_H_ */
