"""Thin ctypes binding of libgvs.so (include/gvs.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  There is no
CPU fallback: if the library is missing or a call fails, this raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgvs.so")

GVS_OK = 0
MAX_VIEWS = 32
_lock = threading.Lock()
_lib = None


class GvsError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


class GvsCamera(ctypes.Structure):
    """Mirror of gvs_camera."""
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


GVS_F32, GVS_F16, GVS_BF16, GVS_U8 = 0, 1, 2, 3


class GvsRefineParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("depth_dtype", ctypes.c_int32)]


class GvsRefineSoftParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_float), ("lambda_t", ctypes.c_float), ("depth_dtype", ctypes.c_int32)]


class GvsFuseParams(ctypes.Structure):
    _fields_ = [("num_samples", ctypes.c_int32), ("z_near", ctypes.c_float), ("z_far", ctypes.c_float),
                ("mu", ctypes.c_float), ("weight_const", ctypes.c_float), ("window", ctypes.c_int32),
                ("normalize", ctypes.c_int32), ("depth_dtype", ctypes.c_int32), ("map_dtype", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


class GvsFuseItem(ctypes.Structure):
    _fields_ = [("map", ctypes.c_void_p), ("map_bytes", ctypes.c_size_t), ("target", ctypes.POINTER(GvsCamera)),
                ("fused_depth", ctypes.c_void_p), ("crossing", ctypes.c_void_p)]


class GvsSplatParams(ctypes.Structure):
    _fields_ = [("footprint", ctypes.c_int32), ("max_half_width", ctypes.c_float), ("mu_guide", ctypes.c_float),
                ("depth_dtype", ctypes.c_int32), ("guide_reject", ctypes.c_int32)]


class GvsGaussParams(ctypes.Structure):
    _fields_ = [("scale_px", ctypes.c_float), ("max_radius", ctypes.c_int32), ("depth_dtype", ctypes.c_int32)]


class GvsSphereParams(ctypes.Structure):
    _fields_ = [("z_near", ctypes.c_float), ("z_far", ctypes.c_float), ("mu", ctypes.c_float),
                ("weight_const", ctypes.c_float), ("window", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("min_frac", ctypes.c_float), ("depth_dtype", ctypes.c_int32)]


class GvsSoftSplatParams(ctypes.Structure):
    _fields_ = [("max_half_width", ctypes.c_float), ("mu_band", ctypes.c_float), ("depth_dtype", ctypes.c_int32),
                ("color_dtype", ctypes.c_int32)]


API = {
    # name: (restype, argtypes)
    "gvs_version": (ctypes.c_char_p, []),
    "gvs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gvs_last_error": (ctypes.c_char_p, []),
    "gvs_refine_depth": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int32] * 3 +
                         [ctypes.POINTER(GvsRefineParams), ctypes.c_void_p]),
    "gvs_refine_soft_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 3),
    "gvs_refine_depth_soft": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int32] * 3 +
                              [ctypes.POINTER(GvsRefineSoftParams), ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p]),
    "gvs_select_views": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_int32, ctypes.POINTER(GvsCamera),
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "gvs_fuse_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 3),
    "gvs_fuse_depth": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsFuseParams),
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]),
    "gvs_weight_map": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_fuse_depth_from_map": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_size_t,
                                               ctypes.c_int32,
                                               ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsFuseParams),
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gvs_fuse_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 3),
    "gvs_fuse_depth_backward": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsFuseParams),
                                               ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_splat_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 3),
    "gvs_temporal_weight": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p] + [ctypes.c_int32] * 5 +
                            [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p]),
    "gvs_fuse_depth_temporal": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_size_t,
                                               ctypes.c_int32, ctypes.POINTER(GvsCamera),
                                               ctypes.POINTER(GvsFuseParams)] + [ctypes.c_void_p] * 6),
    "gvs_guided_mask": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int32] * 3 +
                        [ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "gvs_fuse_batch_bytes": (ctypes.c_size_t, [ctypes.c_int32]),
    "gvs_fuse_batch_create": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_int32, ctypes.POINTER(GvsFuseItem),
                                             ctypes.c_int32, ctypes.POINTER(GvsFuseParams), ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "gvs_fuse_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gvs_fuse_batch_destroy": (None, [ctypes.c_void_p]),
    "gvs_soft_splat_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 3),
    "gvs_soft_splat": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsSoftSplatParams)] +
                       [ctypes.c_void_p] * 6 + [ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_soft_splat_backward": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.POINTER(GvsCamera),
                                               ctypes.POINTER(GvsSoftSplatParams)] + [ctypes.c_void_p] * 9),
    "gvs_soft_splat_backward_blended": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p,
                                                       ctypes.c_int32, ctypes.POINTER(GvsCamera),
                                                       ctypes.POINTER(GvsSoftSplatParams)] + [ctypes.c_void_p] * 8),
    "gvs_uniform_blend_loss_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 2),
    "gvs_uniform_blend_loss": (ctypes.c_int, [ctypes.c_int32] * 3 + [ctypes.c_void_p] * 5 +
                               [ctypes.c_float, ctypes.c_float] + [ctypes.c_void_p] * 4 +
                               [ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_uniform_blend_loss_grad": (ctypes.c_int, [ctypes.c_int32] * 2 + [ctypes.c_void_p] * 4 +
                                    [ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_forward_splat": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsSplatParams),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "gvs_gauss_splat_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 5),
    "gvs_gauss_splat": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsGaussParams), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_blend_features": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_int32, ctypes.POINTER(GvsCamera)] +
                           [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "gvs_blend_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32] * 2),
    "gvs_blend": (ctypes.c_int, [ctypes.c_int32] * 3 + [ctypes.c_void_p] * 4 + [ctypes.c_int32] +
                  [ctypes.c_void_p] * 6 + [ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_fuse_depth_sphere": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(GvsCamera), ctypes.POINTER(GvsSphereParams)] +
                              [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.c_void_p]),
    "gvs_debug_bounds_error": (ctypes.c_uint64, []),
    "gvs_take_device_status": (ctypes.c_uint32, []),
    "gvs_forward_splat_noalloc": (ctypes.c_int, [ctypes.POINTER(GvsCamera), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_int32, ctypes.POINTER(GvsCamera),
                                                 ctypes.POINTER(GvsSplatParams), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Load libgvs.so (built in-tree by __graft_entry__.build()); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in API.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(fn, status):
    if status != GVS_OK:
        lib = load()
        raise GvsError(fn, status, lib.gvs_last_error().decode(errors="replace"))


def take_device_status() -> int:
    """Bulk-copy waits that gave up since the last call (0 in normal operation); read after a
    synchronize."""
    return int(load().gvs_take_device_status())


def camera_struct(c) -> GvsCamera:
    """gvs_camera from any object with width, height, fx, fy, cx, cy, R (3x3), t (3)."""
    s = GvsCamera()
    s.width, s.height = int(c.width), int(c.height)
    s.fx, s.fy, s.cx, s.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    R = [float(x) for row in (c.R.tolist() if hasattr(c.R, "tolist") else c.R) for x in
         (row if hasattr(row, "__iter__") else [row])]
    t = [float(x) for x in (c.t.tolist() if hasattr(c.t, "tolist") else c.t)]
    for a in range(9):
        s.R[a] = R[a]
    for a in range(3):
        s.t[a] = t[a]
    return s


def camera_array(cams):
    arr = (GvsCamera * max(1, len(cams)))()
    for k, c in enumerate(cams):
        arr[k] = camera_struct(c)
    return arr


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("gvs: tensors must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("gvs: tensors must be contiguous")
    return t.data_ptr()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def depth_dtype_of(t) -> int:
    """gvs_dtype of a depth tensor (float32 or float16)."""
    if t.dtype == torch.float32:
        return GVS_F32
    if t.dtype == torch.float16:
        return GVS_F16
    raise ValueError(f"gvs: depth must be float32 or float16, got {t.dtype}")


def _want(t, dtype, shape, name):
    if t.dtype != dtype or tuple(t.shape) != tuple(shape):
        raise ValueError(f"gvs: {name} must be {dtype} of shape {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"gvs: {name} must be contiguous")


def _check_views(in_cams, in_depths, per_pixel=()):
    """The C ABI takes every image size from the cameras, so the tensors must match them:
    in_depths [N, H, W], and each (tensor, bytes per pixel, name) of `per_pixel` N H W times
    that many bytes (a packed int32 or a uint8 [..., 4] RGBA image both hold 4)."""
    N = len(in_cams)
    if N == 0:
        return
    H, W = int(in_cams[0].height), int(in_cams[0].width)
    if tuple(in_depths.shape) != (N, H, W):
        raise ValueError(f"gvs: in_depths must have shape {(N, H, W)} (from the cameras), got {tuple(in_depths.shape)}")
    for t, nb, name in per_pixel:
        if t is not None and t.numel() * t.element_size() != N * H * W * nb:
            raise ValueError(f"gvs: {name} must hold {nb} bytes per input pixel ({N * H * W * nb} bytes), "
                             f"got {t.dtype} {tuple(t.shape)}")


def _check_outputs(out, spec):
    """Caller-supplied output tensors must have the dtype and shape the kernels write."""
    for n, (sh, dt) in spec.items():
        if out.get(n) is not None:
            _want(out[n], dt, sh, n)


def _check_refine(rgba_t, rgba_prev, depth_t, depth_state, mask, mask_dtype):
    N, H, W = depth_t.shape
    if tuple(depth_state.shape) != (N, H, W):
        raise ValueError(f"gvs: depth_state must have shape {(N, H, W)}, got {tuple(depth_state.shape)}")
    for t, name in ((rgba_t, "rgba_t"), (rgba_prev, "rgba_prev")):
        if t is not None and t.numel() * t.element_size() != N * H * W * 4:
            raise ValueError(f"gvs: {name} must hold 4 bytes per pixel of {(N, H, W)}, got {t.dtype} {tuple(t.shape)}")
    if mask is not None:
        _want(mask, mask_dtype, (N, H, W), "mask")


def refine_depth(rgba_t, rgba_prev, depth_t, depth_state, mask=None, tau: float = 0.03, stream=None):
    """Sec. 3.2 Eq. 1-2 (binary mask).  rgba_* int32/uint32 [N, H, W] packed RGBA8 (or uint8 [N, H, W, 4]);
    depth_t, depth_state float32 [N, H, W] (depth_state updated in place); mask uint8 [N, H, W] or None."""
    lib = load()
    N, H, W = depth_t.shape
    if depth_state.dtype != depth_t.dtype:
        raise ValueError("gvs: depth_t and depth_state must share a dtype")
    _check_refine(rgba_t, rgba_prev, depth_t, depth_state, mask, torch.uint8)
    p = GvsRefineParams(float(tau), depth_dtype_of(depth_t))
    st = lib.gvs_refine_depth(_ptr(rgba_t), _ptr(rgba_prev), _ptr(depth_t), _ptr(depth_state), _ptr(mask),
                              N, W, H, ctypes.byref(p), _stream(stream))
    _check("gvs_refine_depth", st)
    return depth_state, mask


def refine_depth_soft(rgba_t, rgba_prev, depth_t, depth_state, mask=None, beta=0.6, lambda_t=0.7, ws=None,
                      stream=None):
    """Sec. 3.2 Eq. 1-2 as printed (soft mask at quarter resolution, max-pool, bilinear).
    depth_state (float32/float16 [N, H, W]) is updated in place; mask: float32 [N, H, W] or None."""
    lib = load()
    N, H, W = depth_t.shape
    _check_refine(rgba_t, rgba_prev, depth_t, depth_state, mask, torch.float32)
    if ws is None:
        ws = workspace(int(lib.gvs_refine_soft_workspace_bytes(N, W, H)), depth_t.device)
    p = GvsRefineSoftParams(float(beta), float(lambda_t), depth_dtype_of(depth_t))
    st = lib.gvs_refine_depth_soft(_ptr(rgba_t), _ptr(rgba_prev), _ptr(depth_t), _ptr(depth_state), _ptr(mask),
                                   N, W, H, ctypes.byref(p), _ptr(ws), ws.numel(), _stream(stream))
    _check("gvs_refine_depth_soft", st)
    return depth_state, mask


def select_views(in_cams, target, k):
    """Indices of the k input cameras closest to the target (host only)."""
    lib = load()
    out = (ctypes.c_int32 * int(k))()
    st = lib.gvs_select_views(camera_array(in_cams), len(in_cams), ctypes.byref(camera_struct(target)), int(k), out)
    _check("gvs_select_views", st)
    return list(out)


def fuse_workspace_bytes(n_views, width, height) -> int:
    return int(load().gvs_fuse_workspace_bytes(n_views, width, height))


def soft_splat_workspace_bytes(n_views, target_width, target_height) -> int:
    return int(load().gvs_soft_splat_workspace_bytes(n_views, target_width, target_height))


def splat_workspace_bytes(n_views, target_width, target_height) -> int:
    return int(load().gvs_splat_workspace_bytes(n_views, target_width, target_height))


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Caller-owned workspace (torch's allocator returns 256-byte aligned blocks)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def fuse_depth(in_cams, in_depths, target, num_samples, z_near, z_far, mu, weight_const=0.001, window=7,
               normalize=False, fused=None, crossing=None, ws=None, want_crossing=True, map_half=False, variant=0,
               stream=None):
    """Supplement A.1 / Eq. 3.  in_depths float32 [N, H, W] on the GPU.
    Returns (fused float32 [Ht, Wt], crossing int16 [Ht, Wt] or None)."""
    lib = load()
    N = len(in_cams)
    dev = in_depths.device
    if fused is None:
        fused = torch.empty((target.height, target.width), dtype=torch.float32, device=dev)
    if crossing is None and want_crossing:
        crossing = torch.empty((target.height, target.width), dtype=torch.int16, device=dev)
    _check_views(in_cams, in_depths)
    _want(fused, torch.float32, (target.height, target.width), "fused")
    if crossing is not None:
        _want(crossing, torch.int16, (target.height, target.width), "crossing")
    H, W = (in_depths.shape[1], in_depths.shape[2]) if N else (0, 0)
    need = fuse_workspace_bytes(N, W, H)
    if ws is None:
        ws = workspace(need, dev)
    p = GvsFuseParams(int(num_samples), float(z_near), float(z_far), float(mu), float(weight_const), int(window),
                      int(bool(normalize)), depth_dtype_of(in_depths) if N else GVS_F32,
                      GVS_F16 if map_half else GVS_F32, int(variant))
    st = lib.gvs_fuse_depth(camera_array(in_cams), _ptr(in_depths), N, ctypes.byref(camera_struct(target)),
                            ctypes.byref(p), _ptr(fused), _ptr(crossing), _ptr(ws), ws.numel(), _stream(stream))
    _check("gvs_fuse_depth", st)
    return fused, crossing


def fuse_depth_backward(in_cams, in_depths, target, num_samples, z_near, z_far, mu, ws, crossing, grad_fused,
                        weight_const=0.001, window=7, map_half=False, grad_depths=None, bwd_ws=None, stream=None):
    """Adjoint of fuse_depth: gradient w.r.t. in_depths (float32 [N, H, W]).  `ws` is the forward's map."""
    lib = load()
    N = len(in_cams)
    _check_views(in_cams, in_depths)
    _want(crossing, torch.int16, (target.height, target.width), "crossing")
    H, W = (in_depths.shape[1], in_depths.shape[2]) if N else (0, 0)
    if grad_depths is None:
        grad_depths = torch.empty(in_depths.shape, dtype=torch.float32, device=in_depths.device)
    if bwd_ws is None:
        bwd_ws = workspace(int(lib.gvs_fuse_backward_workspace_bytes(N, W, H)), in_depths.device)
    grad_fused = grad_fused.contiguous().to(torch.float32)
    _want(grad_fused, torch.float32, (target.height, target.width), "grad_fused")
    _want(grad_depths, torch.float32, tuple(in_depths.shape), "grad_depths")
    p = GvsFuseParams(int(num_samples), float(z_near), float(z_far), float(mu), float(weight_const), int(window), 0,
                      depth_dtype_of(in_depths) if N else GVS_F32, GVS_F16 if map_half else GVS_F32)
    st = lib.gvs_fuse_depth_backward(camera_array(in_cams), _ptr(in_depths), N, ctypes.byref(camera_struct(target)),
                                     ctypes.byref(p), _ptr(ws), ws.numel() * ws.element_size(), _ptr(crossing),
                                     _ptr(grad_fused), _ptr(grad_depths), _ptr(bwd_ws),
                                     bwd_ws.numel() * bwd_ws.element_size(), _stream(stream))
    _check("gvs_fuse_depth_backward", st)
    return grad_depths


class FuseDepth(torch.autograd.Function):
    """Differentiable image-based TSDF fusion: fused = FuseDepth.apply(in_depths, cams, target, cfg).

    cfg: dict(num_samples, z_near, z_far, mu[, weight_const, window, variant]).  The backward
    is gvs_fuse_depth_backward (through the clamped signed distances and the
    confidence weights; the crossing index itself is piecewise constant)."""

    @staticmethod
    def forward(ctx, in_depths, in_cams, target, cfg):
        wc, win = cfg.get("weight_const", 0.001), cfg.get("window", 7)
        N, H, W = in_depths.shape
        ws = workspace(fuse_workspace_bytes(N, W, H), in_depths.device)
        fused, crossing = fuse_depth(in_cams, in_depths, target, cfg["num_samples"], cfg["z_near"], cfg["z_far"],
                                     cfg["mu"], weight_const=wc, window=win, ws=ws, variant=cfg.get("variant", 0))
        ctx.save_for_backward(in_depths, ws, crossing)
        ctx.cams, ctx.target, ctx.cfg = in_cams, target, cfg
        ctx.mark_non_differentiable(crossing)
        return fused, crossing

    @staticmethod
    def backward(ctx, grad_fused, grad_crossing):
        in_depths, ws, crossing = ctx.saved_tensors
        cfg = ctx.cfg
        g = fuse_depth_backward(ctx.cams, in_depths, ctx.target, cfg["num_samples"], cfg["z_near"], cfg["z_far"],
                                cfg["mu"], ws, crossing, grad_fused, weight_const=cfg.get("weight_const", 0.001),
                                window=cfg.get("window", 7))
        return g, None, None, None


def weight_map(in_depths, mu, weight_const=0.001, window=7, ws=None, map_half=False, stream=None):
    """Stage 1 of fusion: the map (packed (depth, weight) float2 [N, H, W] first, then depth-bound tiles),
    written into the uint8 buffer `ws`."""
    lib = load()
    N, H, W = in_depths.shape
    if ws is None:
        ws = workspace(fuse_workspace_bytes(N, W, H), in_depths.device)
    st = lib.gvs_weight_map(_ptr(in_depths), depth_dtype_of(in_depths), N, W, H, float(mu), float(weight_const),
                            int(window), GVS_F16 if map_half else GVS_F32, _ptr(ws), ws.numel() * ws.element_size(),
                            _stream(stream))
    _check("gvs_weight_map", st)
    return ws


def fuse_depth_sphere(in_cams, in_depths, target, z_near, z_far, mu, weight_const=0.001, window=7, max_steps=1024,
                      min_frac=0.0625, fused=None, evals=None, ws=None, stream=None):
    """Supplement A.1's sphere-tracing raymarch (0.8 s steps, three bisections).
    Returns (fused float32 [Ht, Wt] (0: no crossing), evals int32 [Ht, Wt])."""
    lib = load()
    N = len(in_cams)
    dev = in_depths.device
    shape = (target.height, target.width)
    if fused is None:
        fused = torch.empty(shape, dtype=torch.float32, device=dev)
    if evals is None:
        evals = torch.empty(shape, dtype=torch.int32, device=dev)
    _check_views(in_cams, in_depths)
    _want(fused, torch.float32, shape, "fused")
    _want(evals, torch.int32, shape, "evals")
    H, W = (in_depths.shape[1], in_depths.shape[2]) if N else (0, 0)
    if ws is None:
        ws = workspace(fuse_workspace_bytes(N, W, H), dev)
    p = GvsSphereParams(float(z_near), float(z_far), float(mu), float(weight_const), int(window), int(max_steps),
                        float(min_frac), depth_dtype_of(in_depths) if N else GVS_F32)
    st = lib.gvs_fuse_depth_sphere(camera_array(in_cams), _ptr(in_depths), N, ctypes.byref(camera_struct(target)),
                                   ctypes.byref(p), _ptr(fused), _ptr(evals), _ptr(ws), ws.numel(), _stream(stream))
    _check("gvs_fuse_depth_sphere", st)
    return fused, evals


def fuse_depth_from_map(in_cams, dw_map, shape, target, num_samples, z_near, z_far, mu, normalize=False,
                        fused=None, crossing=None, want_crossing=True, map_half=False, variant=0, stream=None):
    """Stage 2 of fusion reading a map from weight_map(); `shape` = (N, H, W) of the inputs."""
    lib = load()
    N = len(in_cams)
    dev = dw_map.device
    if fused is None:
        fused = torch.empty((target.height, target.width), dtype=torch.float32, device=dev)
    if crossing is None and want_crossing:
        crossing = torch.empty((target.height, target.width), dtype=torch.int16, device=dev)
    _want(fused, torch.float32, (target.height, target.width), "fused")
    if crossing is not None:
        _want(crossing, torch.int16, (target.height, target.width), "crossing")
    if N and tuple(shape) != (N, int(in_cams[0].height), int(in_cams[0].width)):
        raise ValueError(f"gvs: shape {tuple(shape)} does not match the {N} cameras")
    p = GvsFuseParams(int(num_samples), float(z_near), float(z_far), float(mu), 0.001, 7, int(bool(normalize)),
                      GVS_F32, GVS_F16 if map_half else GVS_F32, int(variant))
    st = lib.gvs_fuse_depth_from_map(camera_array(in_cams), _ptr(dw_map), dw_map.numel() * dw_map.element_size(), N,
                                     ctypes.byref(camera_struct(target)),
                                     ctypes.byref(p), _ptr(fused), _ptr(crossing), _stream(stream))
    _check("gvs_fuse_depth_from_map", st)
    return fused, crossing


def forward_splat(in_cams, in_depths, in_rgba, target, fused=None, footprint=True, max_half_width=2.0,
                  mu_guide=0.04, outputs=None, ws=None, want=("warped_rgba", "warped_depth", "alpha", "guided"),
                  guide_reject=False, stream=None):
    """Sec. 3.1 / Supplement A.3.  in_depths float32 [N, H, W]; in_rgba int32 [N, H, W] packed RGBA8.
    Returns dict of [N, Ht, Wt] tensors: winner int32, warped_rgba int32, warped_depth float32,
    alpha uint8, guided uint8 (guided only when `fused` is given).  guide_reject: candidates in
    front of fused - mu_guide take no part in the depth test (needs `fused`)."""
    lib = load()
    N = len(in_cams)
    dev = in_depths.device
    shape = (N, target.height, target.width)
    out = dict(outputs or {})
    dtypes = {"winner": torch.int32, "warped_rgba": torch.int32, "warped_depth": torch.float32,
              "alpha": torch.uint8, "guided": torch.uint8}
    names = ["winner"] + [n for n in want if n != "guided" or fused is not None]
    _check_views(in_cams, in_depths, [(in_rgba, 4, "in_rgba")])
    _check_outputs(out, {n: (shape, dt) for n, dt in dtypes.items()})
    if fused is not None:
        _want(fused, torch.float32, shape[1:], "fused")
    for n in names:
        if n not in out:
            out[n] = torch.empty(shape, dtype=dtypes[n], device=dev)
    if ws is None:
        ws = workspace(splat_workspace_bytes(N, target.width, target.height), dev)
    p = GvsSplatParams(int(bool(footprint)), float(max_half_width), float(mu_guide),
                       depth_dtype_of(in_depths) if N else GVS_F32, int(bool(guide_reject)))
    st = lib.gvs_forward_splat(camera_array(in_cams), _ptr(in_depths), _ptr(in_rgba), N,
                               ctypes.byref(camera_struct(target)), ctypes.byref(p), _ptr(fused),
                               _ptr(out["winner"]), _ptr(out.get("warped_rgba")), _ptr(out.get("warped_depth")),
                               _ptr(out.get("alpha")), _ptr(out.get("guided")), _ptr(ws), ws.numel(),
                               _stream(stream))
    _check("gvs_forward_splat", st)
    return out


def _color_dtype_of(t) -> int:
    if t.dtype == torch.float32:
        return GVS_F32
    if t.dtype == torch.bfloat16:
        return GVS_BF16
    raise ValueError(f"gvs: soft-splat colour must be float32 or bfloat16, got {t.dtype}")


def gauss_splat_workspace_bytes(width, height, target_width, target_height, max_radius=8) -> int:
    return int(load().gvs_gauss_splat_workspace_bytes(width, height, target_width, target_height, max_radius))


def gauss_splat(in_cams, in_depths, in_rgba, target, scale_px=0.5, max_radius=8, color=None, depth=None, ws=None,
                stream=None):
    """Pixel-sized Gaussians alpha-composited per view (Sec. 3.1, Supplement A.3).
    in_depths float32/float16 [N, H, W]; in_rgba int32 [N, H, W] packed RGBA8.
    Returns (color float32 [N, Ht, Wt, 4] premultiplied rgb + opacity, depth float32 [N, Ht, Wt])."""
    lib = load()
    N = len(in_cams)
    dev = in_depths.device
    shape = (N, target.height, target.width)
    if color is None:
        color = torch.empty(shape + (4,), dtype=torch.float32, device=dev)
    if depth is None:
        depth = torch.empty(shape, dtype=torch.float32, device=dev)
    _want(color, torch.float32, shape + (4,), "color")
    _want(depth, torch.float32, shape, "depth")
    if N == 0:
        return color, depth
    _check_views(in_cams, in_depths, [(in_rgba, 4, "in_rgba")])
    H, W = in_depths.shape[1], in_depths.shape[2]
    if ws is None:
        ws = workspace(gauss_splat_workspace_bytes(W, H, target.width, target.height, max_radius), dev)
    p = GvsGaussParams(float(scale_px), int(max_radius), depth_dtype_of(in_depths))
    st = lib.gvs_gauss_splat(camera_array(in_cams), _ptr(in_depths), _ptr(in_rgba), N,
                             ctypes.byref(camera_struct(target)), ctypes.byref(p), _ptr(color), _ptr(depth), _ptr(ws),
                             ws.numel(), _stream(stream))
    _check("gvs_gauss_splat", st)
    return color, depth


_FEATURE_DTYPES = {torch.float32: GVS_F32, torch.float16: GVS_F16, torch.bfloat16: GVS_BF16}


def blend_features(in_cams, target, warped_rgba, warped_depth, alpha, fused, dtype=torch.float32, out=None,
                   stream=None):
    """The blending network's (9K + 1) x Ht x Wt input (Sec. 3.3 and the supplement's list),
    from the splat outputs (warped_rgba int32, warped_depth float32, alpha uint8, each
    [K, Ht, Wt]) and the TSDF depth fused float32 [Ht, Wt]."""
    lib = load()
    K = len(in_cams)
    if out is None:
        out = torch.empty((9 * K + 1, target.height, target.width), dtype=dtype, device=fused.device)
    sh = (K, target.height, target.width)
    _want(warped_rgba, warped_rgba.dtype, sh, "warped_rgba")
    if warped_rgba.element_size() != 4:
        raise ValueError("gvs: warped_rgba must be packed 32-bit RGBA")
    _want(warped_depth, torch.float32, sh, "warped_depth")
    _want(alpha, torch.uint8, sh, "alpha")
    _want(fused, torch.float32, sh[1:], "fused")
    _want(out, out.dtype, (9 * K + 1,) + sh[1:], "out")
    st = lib.gvs_blend_features(camera_array(in_cams), K, ctypes.byref(camera_struct(target)), _ptr(warped_rgba),
                                _ptr(warped_depth), _ptr(alpha), _ptr(fused), _FEATURE_DTYPES[out.dtype], _ptr(out),
                                _stream(stream))
    _check("gvs_blend_features", st)
    return out


def blend(warped_rgba, alpha, warped_depth, fused, w, w_bg, i_bg, image=None, l_depth=None, ws=None, stream=None):
    """Eqs. 4-5 and L_Depth.  w [K, Ht, Wt], w_bg [Ht, Wt], i_bg [3, Ht, Wt], float32 or bfloat16
    (contiguous planes, e.g. slices of the network output).  Returns (image float32 [3, Ht, Wt],
    L_Depth float64 scalar tensor on the device)."""
    lib = load()
    K, Ht, Wt = warped_rgba.shape
    dev = fused.device
    if image is None:
        image = torch.empty((3, Ht, Wt), dtype=torch.float32, device=dev)
    if l_depth is None:
        l_depth = torch.empty((), dtype=torch.float64, device=dev)
    if ws is None:
        ws = workspace(int(lib.gvs_blend_workspace_bytes(Wt, Ht)), dev)
    wdt = {torch.float32: GVS_F32, torch.bfloat16: GVS_BF16}[w.dtype]
    if warped_rgba.element_size() != 4:
        raise ValueError("gvs: warped_rgba must be packed 32-bit RGBA")
    _want(alpha, torch.uint8, (K, Ht, Wt), "alpha")
    _want(warped_depth, torch.float32, (K, Ht, Wt), "warped_depth")
    _want(fused, torch.float32, (Ht, Wt), "fused")
    _want(w, w.dtype, (K, Ht, Wt), "w")
    _want(w_bg, w.dtype, (Ht, Wt), "w_bg")
    _want(i_bg, w.dtype, (3, Ht, Wt), "i_bg")
    _want(image, torch.float32, (3, Ht, Wt), "image")
    st = lib.gvs_blend(K, Wt, Ht, _ptr(warped_rgba), _ptr(alpha), _ptr(warped_depth), _ptr(fused), wdt, _ptr(w),
                       _ptr(w_bg), _ptr(i_bg), _ptr(image), _ptr(l_depth), _ptr(ws), ws.numel(), _stream(stream))
    _check("gvs_blend", st)
    return image, l_depth


def soft_splat(in_cams, in_depths, in_color, target, max_half_width=2.0, mu_band=0.04, outputs=None, ws=None,
               stream=None):
    """Differentiable colour splat.  in_color [N, H, W, 4] float32 or bfloat16 in [0, 1].
    Returns dict: winner int32, color float32 [N, Ht, Wt, 4], depth float32, wsum float32, alpha uint8."""
    lib = load()
    N = len(in_cams)
    dev = in_depths.device
    shape = (N, target.height, target.width)
    out = dict(outputs or {})
    spec = {"winner": (shape, torch.int32), "color": (shape + (4,), torch.float32), "depth": (shape, torch.float32),
            "wsum": (shape, torch.float32), "alpha": (shape, torch.uint8)}
    _check_views(in_cams, in_depths)
    if N and tuple(in_color.shape) != tuple(in_depths.shape) + (4,):
        raise ValueError(f"gvs: in_color must have shape {tuple(in_depths.shape) + (4,)}, got {tuple(in_color.shape)}")
    _check_outputs(out, spec)
    for n, (sh, dt) in spec.items():
        if n not in out:
            out[n] = torch.empty(sh, dtype=dt, device=dev)
    if ws is None:
        ws = workspace(int(lib.gvs_soft_splat_workspace_bytes(N, target.width, target.height)), dev)
    p = GvsSoftSplatParams(float(max_half_width), float(mu_band), depth_dtype_of(in_depths) if N else GVS_F32,
                           _color_dtype_of(in_color) if N else GVS_F32)
    st = lib.gvs_soft_splat(camera_array(in_cams), _ptr(in_depths), _ptr(in_color), N,
                            ctypes.byref(camera_struct(target)), ctypes.byref(p), _ptr(out["winner"]),
                            _ptr(out["color"]), _ptr(out["depth"]), _ptr(out["wsum"]), _ptr(out["alpha"]), _ptr(ws),
                            ws.numel() * ws.element_size(), _stream(stream))
    _check("gvs_soft_splat", st)
    return out


def soft_splat_backward(in_cams, in_depths, in_color, target, fwd, grad_color, grad_depth=None, max_half_width=2.0,
                        mu_band=0.04, stream=None):
    """Adjoint of soft_splat: (grad w.r.t. in_depths float32 [N, H, W], w.r.t. in_color float32 [N, H, W, 4])."""
    lib = load()
    N = len(in_cams)
    _check_views(in_cams, in_depths)
    shape = (N, target.height, target.width)
    if N and tuple(in_color.shape) != tuple(in_depths.shape) + (4,):
        raise ValueError(f"gvs: in_color must have shape {tuple(in_depths.shape) + (4,)}, got {tuple(in_color.shape)}")
    _check_outputs(fwd, {"winner": (shape, torch.int32), "color": (shape + (4,), torch.float32),
                         "depth": (shape, torch.float32), "wsum": (shape, torch.float32)})
    gd = torch.empty(in_depths.shape, dtype=torch.float32, device=in_depths.device)
    gc = torch.empty(tuple(in_color.shape[:3]) + (4,), dtype=torch.float32, device=in_depths.device)
    grad_color = grad_color.contiguous().to(torch.float32)
    _want(grad_color, torch.float32, shape + (4,), "grad_color")
    if grad_depth is not None:
        grad_depth = grad_depth.contiguous().to(torch.float32)
        _want(grad_depth, torch.float32, shape, "grad_depth")
    p = GvsSoftSplatParams(float(max_half_width), float(mu_band), depth_dtype_of(in_depths) if N else GVS_F32,
                           _color_dtype_of(in_color) if N else GVS_F32)
    st = lib.gvs_soft_splat_backward(camera_array(in_cams), _ptr(in_depths), _ptr(in_color), N,
                                     ctypes.byref(camera_struct(target)), ctypes.byref(p), _ptr(fwd["winner"]),
                                     _ptr(fwd["color"]), _ptr(fwd["depth"]), _ptr(fwd["wsum"]), _ptr(grad_color),
                                     _ptr(grad_depth), _ptr(gd), _ptr(gc), _stream(stream))
    _check("gvs_soft_splat_backward", st)
    return gd, gc


def soft_splat_backward_blended(in_cams, in_depths, in_color, target, fwd, grad_pixel, max_half_width=2.0,
                                mu_band=0.04, stream=None):
    """Adjoint of soft_splat for upstream gradients shared by the views per target pixel:
    grad_pixel float32 [Ht, Wt, 4] (d/d colour RGB, d/d warped depth).  Returns the gradients
    w.r.t. in_depths [N, H, W] and in_color [N, H, W, 4]."""
    lib = load()
    N = len(in_cams)
    _check_views(in_cams, in_depths)
    shape = (N, target.height, target.width)
    if N and tuple(in_color.shape) != tuple(in_depths.shape) + (4,):
        raise ValueError(f"gvs: in_color must have shape {tuple(in_depths.shape) + (4,)}, got {tuple(in_color.shape)}")
    _check_outputs(fwd, {"winner": (shape, torch.int32), "color": (shape + (4,), torch.float32),
                         "depth": (shape, torch.float32), "wsum": (shape, torch.float32)})
    _want(grad_pixel, torch.float32, (target.height, target.width, 4), "grad_pixel")
    gd = torch.empty(in_depths.shape, dtype=torch.float32, device=in_depths.device)
    gc = torch.empty(tuple(in_color.shape[:3]) + (4,), dtype=torch.float32, device=in_depths.device)
    p = GvsSoftSplatParams(float(max_half_width), float(mu_band), depth_dtype_of(in_depths) if N else GVS_F32,
                           _color_dtype_of(in_color) if N else GVS_F32)
    st = lib.gvs_soft_splat_backward_blended(camera_array(in_cams), _ptr(in_depths), _ptr(in_color), N,
                                             ctypes.byref(camera_struct(target)), ctypes.byref(p),
                                             _ptr(fwd["winner"]), _ptr(fwd["color"]), _ptr(fwd["depth"]),
                                             _ptr(fwd["wsum"]), _ptr(grad_pixel), _ptr(gd), _ptr(gc), _stream(stream))
    _check("gvs_soft_splat_backward_blended", st)
    return gd, gc


def uniform_blend_loss(color, alpha, warped_depth, fused, gt, w_l1=0.8, w_depth=0.1, want_grad=True, ws=None,
                       stream=None):
    """Sec. 3.3's loss on the uniform blend of the views (gvs_uniform_blend_loss).
    color float32 [N, Ht, Wt, 4], alpha uint8 [N, Ht, Wt], warped_depth float32 [N, Ht, Wt],
    fused float32 [Ht, Wt], gt float32 [Ht, Wt, 3].  Returns (loss float64 [3] = L, L1, L_Depth on
    the device, grad_pixel float32 [Ht, Wt, 4] or None, grad_fused float32 [Ht, Wt] or None).
    ws: a workspace of blend_loss_workspace_bytes(Ht, Wt) bytes to keep for
    uniform_blend_loss_grad (a fresh one when None)."""
    lib = load()
    N, Ht, Wt = alpha.shape
    dev = alpha.device
    _want(color, torch.float32, (N, Ht, Wt, 4), "color")
    _want(alpha, torch.uint8, (N, Ht, Wt), "alpha")
    _want(warped_depth, torch.float32, (N, Ht, Wt), "warped_depth")
    _want(fused, torch.float32, (Ht, Wt), "fused")
    _want(gt, torch.float32, (Ht, Wt, 3), "gt")
    loss = torch.empty(3, dtype=torch.float64, device=dev)
    gp = torch.empty((Ht, Wt, 4), dtype=torch.float32, device=dev) if want_grad else None
    gf = torch.empty((Ht, Wt), dtype=torch.float32, device=dev) if want_grad else None
    if ws is None:
        ws = workspace(blend_loss_workspace_bytes(Ht, Wt), dev)
    st = lib.gvs_uniform_blend_loss(N, Wt, Ht, _ptr(color), _ptr(alpha), _ptr(warped_depth), _ptr(fused), _ptr(gt),
                                    float(w_l1), float(w_depth), _ptr(loss), _ptr(gp), _ptr(gf), _ptr(ws),
                                    ws.numel(), _stream(stream))
    _check("gvs_uniform_blend_loss", st)
    return loss, gp, gf


def blend_loss_workspace_bytes(Ht, Wt):
    return int(load().gvs_uniform_blend_loss_workspace_bytes(Wt, Ht))


def uniform_blend_loss_grad(ws, Ht, Wt, grad_loss=None, stream=None):
    """gvs_uniform_blend_loss_grad: the gradient of the loss the last uniform_blend_loss on ws
    computed, times grad_loss (a float32 scalar tensor on the device; None for 1).
    Returns (grad_pixel float32 [Ht, Wt, 4], grad_fused float32 [Ht, Wt])."""
    lib = load()
    dev = ws.device
    if grad_loss is not None:
        if grad_loss.dtype != torch.float32 or grad_loss.numel() != 1 or grad_loss.device != dev:
            raise ValueError("grad_loss: one float32 value on the workspace's device")
        grad_loss = grad_loss.contiguous()
    gp = torch.empty((Ht, Wt, 4), dtype=torch.float32, device=dev)
    gf = torch.empty((Ht, Wt), dtype=torch.float32, device=dev)
    st = lib.gvs_uniform_blend_loss_grad(Wt, Ht, _ptr(grad_loss), _ptr(gp), _ptr(gf), _ptr(ws), ws.numel(),
                                         _stream(stream))
    _check("gvs_uniform_blend_loss_grad", st)
    return gp, gf


class SoftSplatBlendLoss(torch.autograd.Function):
    """L = SoftSplatBlendLoss.apply(in_depths, in_color, fused, cams, target, gt, cfg): the
    differentiable splat of every view, blended with uniform weights and scored against gt by
    Sec. 3.3's w_l1 L1 + w_depth L_Depth (cfg: mu_band, max_half_width=2.0, w_l1=0.8,
    w_depth=0.1).  Returns L as a float32 scalar tensor; the gradient flows to in_depths and
    in_color (through the splat's adjoint) and to fused."""

    @staticmethod
    def forward(ctx, in_depths, in_color, fused, in_cams, target, gt, cfg):
        mhw = cfg.get("max_half_width", 2.0)
        fwd = soft_splat(in_cams, in_depths, in_color, target, mhw, cfg["mu_band"])
        Ht, Wt = target.height, target.width
        ws = workspace(blend_loss_workspace_bytes(Ht, Wt), in_depths.device)
        # the loss now; its gradient in backward, from the signs kept in ws, times the upstream
        loss, _, _ = uniform_blend_loss(fwd["color"], fwd["alpha"], fwd["depth"], fused.detach().contiguous(), gt,
                                        cfg.get("w_l1", 0.8), cfg.get("w_depth", 0.1), want_grad=False, ws=ws)
        ctx.save_for_backward(in_depths, in_color, fwd["winner"], fwd["color"], fwd["depth"], fwd["wsum"], ws)
        ctx.cams, ctx.target, ctx.cfg = in_cams, target, cfg
        return loss[0].to(torch.float32)

    @staticmethod
    def backward(ctx, g):
        in_depths, in_color, winner, color, depth, wsum, ws = ctx.saved_tensors
        gp, gf = uniform_blend_loss_grad(ws, ctx.target.height, ctx.target.width, g.to(torch.float32))
        fwd = {"winner": winner, "color": color, "depth": depth, "wsum": wsum}
        gd, gc = soft_splat_backward_blended(ctx.cams, in_depths, in_color, ctx.target, fwd, gp,
                                             ctx.cfg.get("max_half_width", 2.0), ctx.cfg["mu_band"])
        return gd, gc.to(in_color.dtype), gf, None, None, None, None


class SoftSplat(torch.autograd.Function):
    """color, depth, alpha = SoftSplat.apply(in_depths, in_color, cams, target, cfg);
    cfg: dict(max_half_width=2.0, mu_band).  Gradients flow to in_depths and in_color."""

    @staticmethod
    def forward(ctx, in_depths, in_color, in_cams, target, cfg):
        fwd = soft_splat(in_cams, in_depths, in_color, target, cfg.get("max_half_width", 2.0), cfg["mu_band"])
        ctx.save_for_backward(in_depths, in_color, fwd["winner"], fwd["color"], fwd["depth"], fwd["wsum"])
        ctx.cams, ctx.target, ctx.cfg = in_cams, target, cfg
        ctx.mark_non_differentiable(fwd["alpha"])
        return fwd["color"], fwd["depth"], fwd["alpha"]

    @staticmethod
    def backward(ctx, g_color, g_depth, g_alpha):
        in_depths, in_color, winner, color, depth, wsum = ctx.saved_tensors
        fwd = {"winner": winner, "color": color, "depth": depth, "wsum": wsum}
        gd, gc = soft_splat_backward(ctx.cams, in_depths, in_color, ctx.target, fwd,
                                     g_color if g_color is not None else torch.zeros_like(color), g_depth,
                                     ctx.cfg.get("max_half_width", 2.0), ctx.cfg["mu_band"])
        return gd, gc.to(in_color.dtype), None, None, None


class FuseBatch:
    """Batched fusion of many (map, target) items in one persistent launch (gvs_fuse_batch_*).

    items: list of (map_tensor, target_camera, fused_out [Ht, Wt] float32, crossing_out int16 or None).
    Create outside any stream capture (it copies the item table); launch() may be captured."""

    def __init__(self, in_cams, items, num_samples, z_near, z_far, mu, normalize=False, map_half=False, variant=0):
        lib = load()
        self.lib = lib
        self._keep = items  # the tensors must outlive the batch
        self._targets = [camera_struct(t) for _, t, _, _ in items]
        arr = (GvsFuseItem * len(items))()
        for n, (m, t, f, c) in enumerate(items):
            _want(f, torch.float32, (t.height, t.width), f"items[{n}] fused")
            if c is not None:
                _want(c, torch.int16, (t.height, t.width), f"items[{n}] crossing")
            arr[n] = GvsFuseItem(_ptr(m), m.numel() * m.element_size(), ctypes.pointer(self._targets[n]), _ptr(f),
                                 _ptr(c))
        p = GvsFuseParams(int(num_samples), float(z_near), float(z_far), float(mu), 0.001, 7, int(bool(normalize)),
                          GVS_F32, GVS_F16 if map_half else GVS_F32, int(variant))
        dev = items[0][0].device
        self.table = workspace(int(lib.gvs_fuse_batch_bytes(len(items))), dev)
        h = ctypes.c_void_p()
        st = lib.gvs_fuse_batch_create(camera_array(in_cams), len(in_cams), arr, len(items), ctypes.byref(p),
                                       _ptr(self.table), self.table.numel(), ctypes.byref(h))
        _check("gvs_fuse_batch_create", st)
        self.handle = h

    def launch(self, stream=None):
        _check("gvs_fuse_batch_launch", self.lib.gvs_fuse_batch_launch(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            self.lib.gvs_fuse_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def temporal_weight(masks, winner, w_tmp_prev, w_view_prev, beta_t=1.0, eta=15.0, w_tmp=None, target_mask=None,
                    stream=None):
    """Supplement A.2 temporal fusion weight (see gvs_temporal_weight).  masks float32 or uint8 [N, H, W]."""
    lib = load()
    N, H, W = masks.shape
    Ht, Wt = winner.shape[1:]
    if w_tmp is None:
        w_tmp = torch.empty((Ht, Wt), dtype=torch.float32, device=masks.device)
    _want(winner, torch.int32, (N, Ht, Wt), "winner")
    for t, name in ((w_tmp_prev, "w_tmp_prev"), (w_view_prev, "w_view_prev"), (w_tmp, "w_tmp")):
        _want(t, torch.float32, (Ht, Wt), name)
    if target_mask is not None:
        _want(target_mask, torch.float32, (Ht, Wt), "target_mask")
    md = GVS_U8 if masks.dtype == torch.uint8 else GVS_F32
    st = lib.gvs_temporal_weight(_ptr(masks), md, _ptr(winner), N, W, H, Wt, Ht, _ptr(w_tmp_prev), _ptr(w_view_prev),
                                 float(beta_t), float(eta), _ptr(w_tmp), _ptr(target_mask), _stream(stream))
    _check("gvs_temporal_weight", st)
    return w_tmp


def fuse_depth_temporal(in_cams, dw_map, target, num_samples, z_near, z_far, mu, prev_depth, w_tmp, fused=None,
                        crossing=None, view_weight=None, stream=None):
    """fuse_depth_from_map with the previous output depth as one more input (Supplement A.2)."""
    lib = load()
    N = len(in_cams)
    dev = dw_map.device
    shape = (target.height, target.width)
    if fused is None:
        fused = torch.empty(shape, dtype=torch.float32, device=dev)
    if crossing is None:
        crossing = torch.empty(shape, dtype=torch.int16, device=dev)
    if view_weight is None:
        view_weight = torch.empty(shape, dtype=torch.float32, device=dev)
    for t, dt, name in ((prev_depth, torch.float32, "prev_depth"), (w_tmp, torch.float32, "w_tmp"),
                        (fused, torch.float32, "fused"), (crossing, torch.int16, "crossing"),
                        (view_weight, torch.float32, "view_weight")):
        _want(t, dt, shape, name)
    p = GvsFuseParams(int(num_samples), float(z_near), float(z_far), float(mu), 0.001, 7, 0, GVS_F32, GVS_F32, 0)
    st = lib.gvs_fuse_depth_temporal(camera_array(in_cams), _ptr(dw_map), dw_map.numel(), N,
                                     ctypes.byref(camera_struct(target)), ctypes.byref(p), _ptr(prev_depth),
                                     _ptr(w_tmp), _ptr(fused), _ptr(crossing), _ptr(view_weight), _stream(stream))
    _check("gvs_fuse_depth_temporal", st)
    return fused, crossing, view_weight


def guided_mask(warped_depth, alpha, fused, mu_guide, guided=None, stream=None):
    lib = load()
    N, Ht, Wt = warped_depth.shape
    if guided is None:
        guided = torch.empty((N, Ht, Wt), dtype=torch.uint8, device=warped_depth.device)
    _want(alpha, torch.uint8, (N, Ht, Wt), "alpha")
    _want(fused, torch.float32, (Ht, Wt), "fused")
    _want(guided, torch.uint8, (N, Ht, Wt), "guided")
    st = lib.gvs_guided_mask(_ptr(warped_depth), _ptr(alpha), _ptr(fused), N, Wt, Ht, float(mu_guide), _ptr(guided),
                             _stream(stream))
    _check("gvs_guided_mask", st)
    return guided


class TemporalFusion:
    """Online fused depth with the temporal term (Sec. 3.2, Supplement A.2) for a fixed
    novel viewpoint.  Per frame: splat the views (winners), the temporal weight from the
    splatted difference masks and the previous frame's state, the fusion with the previous
    output as one more input, then the guided mask.  State per target pixel: previous
    fused depth, temporal weight, views' weight at the crossing (all start at 0)."""

    def __init__(self, in_cams, target, num_samples, z_near, z_far, mu, beta_t=1.0, eta=15.0, device="cuda"):
        self.cams, self.target = in_cams, target
        self.cfg = dict(num_samples=num_samples, z_near=z_near, z_far=z_far, mu=mu, beta_t=beta_t, eta=eta)
        shape = (target.height, target.width)
        self.prev = torch.zeros(shape, dtype=torch.float32, device=device)
        self.w_tmp_prev = torch.zeros(shape, dtype=torch.float32, device=device)
        self.w_view_prev = torch.zeros(shape, dtype=torch.float32, device=device)

    def step(self, depths, rgba, masks, ws_map=None):
        c = self.cfg
        m = weight_map(depths, c["mu"], ws=ws_map)
        sp = forward_splat(self.cams, depths, rgba, self.target, fused=None, mu_guide=c["mu"])
        w_tmp = temporal_weight(masks, sp["winner"], self.w_tmp_prev, self.w_view_prev, c["beta_t"], c["eta"])
        fused, crossing, wview = fuse_depth_temporal(self.cams, m, self.target, c["num_samples"], c["z_near"],
                                                     c["z_far"], c["mu"], self.prev, w_tmp)
        sp["guided"] = guided_mask(sp["warped_depth"], sp["alpha"], fused, c["mu"])
        self.prev, self.w_tmp_prev, self.w_view_prev = fused, w_tmp, wview
        return fused, crossing, sp, w_tmp

    _STATE = ("prev", "w_tmp_prev", "w_view_prev")

    def state_dict(self):
        """Checkpoint of the online state (host copies).  With the caller's refined input
        depths it is everything a later frame depends on: restoring both resumes the
        stream bit for bit."""
        return {k: getattr(self, k).cpu() for k in self._STATE}

    def load_state_dict(self, sd):
        dev = self.prev.device
        for k in self._STATE:
            setattr(self, k, sd[k].to(device=dev, dtype=torch.float32).clone())
