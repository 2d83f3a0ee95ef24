"""FP64 CPU oracle (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It is a plain, slow statement of the
method, written from the paper, and shares no code with the CUDA library.
See `oracle/oracle.c` for the passages each function follows and for the
readings taken where the paper is silent.

Parity pins: tests/test_oracle_refine.py, tests/test_oracle_fuse.py,
tests/test_oracle_splat.py (closed forms, invariants, brute force, golden
fixtures under tests/golden/).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_WEIGHT_CONST = 0.001   # Supplement A.1
DEFAULT_WINDOW = 7             # Supplement A.1, w = 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


class _Cam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


def _cam(c) -> _Cam:
    s = _Cam()
    s.width, s.height = int(c.width), int(c.height)
    s.fx, s.fy, s.cx, s.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    R = np.asarray(c.R, np.float64).reshape(9)
    t = np.asarray(c.t, np.float64).reshape(3)
    for a in range(9):
        s.R[a] = R[a]
    for a in range(3):
        s.t[a] = t[a]
    return s


def _cams(cs):
    arr = (_Cam * len(cs))()
    for k, c in enumerate(cs):
        arr[k] = _cam(c)
    return arr


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, dbl, flt = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
            cp = ctypes.POINTER(_Cam)
            lib.orc_refine_depth.argtypes = [i32, i32, i32, vp, vp, vp, vp, flt, vp, vp]
            lib.orc_weight.argtypes = [vp, i32, i32, i32, i32, dbl, dbl, i32]
            lib.orc_weight.restype = dbl
            lib.orc_fuse_depth.argtypes = [cp, vp, i32, cp, i32, dbl, dbl, dbl, dbl, i32, i32, vp, i64,
                                           vp, vp, vp, vp, i32]
            lib.orc_forward_splat.argtypes = [cp, vp, vp, i32, cp, i32, flt, flt, i32, vp, vp, vp, vp, vp, vp, vp,
                                              vp]
            lib.orc_splat_bruteforce.argtypes = [cp, vp, i32, cp, i32, flt, vp]
            lib.orc_fuse_depth_grad.argtypes = [cp, vp, i32, cp, i32, dbl, dbl, dbl, dbl, i32, vp, vp]
            lib.orc_refine_depth_soft.argtypes = [i32, i32, i32, vp, vp, vp, vp, dbl, dbl, vp, vp]
            lib.orc_temporal_weight.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp, dbl, dbl, vp, vp]
            lib.orc_fuse_depth_temporal.argtypes = [cp, vp, i32, cp, i32, dbl, dbl, dbl, dbl, i32, vp, vp, vp, vp,
                                                    vp, vp]
            lib.orc_blend_features.argtypes = [cp, i32, cp, vp, vp, vp, vp, vp]
            lib.orc_blend.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_weight_f32.restype = flt
            lib.orc_weight_f32.argtypes = [vp, i32, i32, i32, i32, flt, flt, i32, flt]
            lib.orc_fuse_depth_sphere.argtypes = [cp, vp, i32, cp, dbl, dbl, dbl, dbl, i32, i32, dbl, vp, vp]
            lib.orc_gauss_splat.argtypes = [cp, vp, vp, i32, cp, flt, i32, vp, i64, vp, vp, vp]
            lib.orc_soft_splat.argtypes = [cp, vp, vp, i32, cp, flt, flt, vp, vp, vp, vp, vp]
            lib.orc_soft_splat_grad.argtypes = [cp, vp, vp, i32, cp, flt, flt, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _threads(n):
    return n if n else min(64, os.cpu_count() or 1)


def refine_depth(rgba_t, rgba_prev, depth_t, state_prev, tau: float = 0.03):
    """Eq. 1-2, binary form.  Arrays [N, H, W(, 4)]; rgba_prev None at t = 0.

    Returns (state_out float32 [N, H, W], mask uint8 [N, H, W])."""
    lib = _load()
    rgba_t = np.ascontiguousarray(rgba_t, np.uint8)
    N, H, W = rgba_t.shape[:3]
    depth_t = np.ascontiguousarray(depth_t, np.float32)
    rp = None if rgba_prev is None else np.ascontiguousarray(rgba_prev, np.uint8)
    sp = None if state_prev is None else np.ascontiguousarray(state_prev, np.float32)
    out = np.empty((N, H, W), np.float32)
    mask = np.empty((N, H, W), np.uint8)
    rc = lib.orc_refine_depth(N, H, W, _ptr(rgba_t), _ptr(rp), _ptr(depth_t), _ptr(sp), ctypes.c_float(tau),
                              _ptr(out), _ptr(mask))
    if rc != 0:
        raise ValueError("orc_refine_depth rejected its arguments")
    return out, mask


def refine_depth_soft(rgba_t, rgba_prev, depth_t, state_prev, beta=0.6, lambda_t=0.7):
    """Eq. 1-2 in the paper's soft form (quarter resolution, 3x3 max-pool, bilinear upsample).

    Returns (state_out float64 [N, H, W], mask float64 [N, H, W])."""
    lib = _load()
    rgba_t = np.ascontiguousarray(rgba_t, np.uint8)
    rgba_prev = np.ascontiguousarray(rgba_prev, np.uint8)
    N, H, W = rgba_t.shape[:3]
    d = np.ascontiguousarray(depth_t, np.float32)
    sp = np.ascontiguousarray(state_prev, np.float32)
    out = np.empty((N, H, W), np.float64)
    mask = np.empty((N, H, W), np.float64)
    rc = lib.orc_refine_depth_soft(N, H, W, _ptr(rgba_t), _ptr(rgba_prev), _ptr(d), _ptr(sp), float(beta),
                                   float(lambda_t), _ptr(out), _ptr(mask))
    if rc != 0:
        raise ValueError("orc_refine_depth_soft rejected its arguments")
    return out, mask


def weight(depth, u: int, v: int, mu: float, weight_const=DEFAULT_WEIGHT_CONST, window=DEFAULT_WINDOW) -> float:
    """Supplement A.1 confidence weight of one view at pixel (u, v)."""
    lib = _load()
    d = np.ascontiguousarray(depth, np.float32)
    H, W = d.shape
    return lib.orc_weight(_ptr(d), H, W, int(u), int(v), float(mu), float(weight_const), int(window))


def fuse_depth(in_cams, depths, target, num_samples, z_near, z_far, mu,
               weight_const=DEFAULT_WEIGHT_CONST, window=DEFAULT_WINDOW, normalize=False,
               pixels=None, threads=None, count_fp64=False):
    """Fused target depth by D uniform samples and the first +/- crossing.

    `pixels`: optional int array [P, 2] of (column, row); default every pixel.
    Returns dict(depth float64, index int32 (-1 none), ambiguous uint8,
    fp64_mismatch int) shaped [Ht, Wt] or [P]."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    if pixels is not None:
        pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        n = pix.shape[0]
        shape = (n,)
    else:
        pix = None
        n = target.width * target.height
        shape = (target.height, target.width)
    out_d = np.empty(n, np.float64)
    out_i = np.empty(n, np.int32)
    out_a = np.empty(n, np.uint8)
    mism = ctypes.c_int64(0)
    rc = lib.orc_fuse_depth(_cams(in_cams), _ptr(depths), len(in_cams), ctypes.byref(_cam(target)),
                            int(num_samples), float(np.float32(z_near)), float(np.float32(z_far)),
                            float(np.float32(mu)), float(weight_const), int(window), int(bool(normalize)),
                            _ptr(pix), n, _ptr(out_d), _ptr(out_i), _ptr(out_a),
                            ctypes.addressof(mism) if count_fp64 else None, _threads(threads))
    if rc != 0:
        raise ValueError("orc_fuse_depth rejected its arguments")
    return {"depth": out_d.reshape(shape), "index": out_i.reshape(shape), "ambiguous": out_a.reshape(shape),
            "fp64_mismatch": int(mism.value)}


def temporal_weight(masks, winner, w_tmp_prev, w_view_prev, beta_t=1.0, eta=15.0):
    """Supplement A.2: target-view difference mask (max over views at the z-buffer winners)
    and the temporal fusion weight.  masks float [N, H, W]; winner int32 [N, Ht, Wt].
    Returns (w_tmp float64 [Ht, Wt], mask float64 [Ht, Wt])."""
    lib = _load()
    masks = np.ascontiguousarray(masks, np.float32)
    winner = np.ascontiguousarray(winner, np.int32)
    N, H, W = masks.shape
    Ht, Wt = winner.shape[1:]
    wp = np.ascontiguousarray(w_tmp_prev, np.float32)
    wv = np.ascontiguousarray(w_view_prev, np.float32)
    out = np.empty((Ht, Wt), np.float64)
    m = np.empty((Ht, Wt), np.float64)
    rc = lib.orc_temporal_weight(_ptr(masks), _ptr(winner), N, W, H, Wt, Ht, _ptr(wp), _ptr(wv), float(beta_t),
                                 float(eta), _ptr(out), _ptr(m))
    if rc != 0:
        raise ValueError("orc_temporal_weight rejected its arguments")
    return out, m


def fuse_depth_temporal(in_cams, depths, target, num_samples, z_near, z_far, mu, tmp_depth, tmp_weight,
                        weight_const=DEFAULT_WEIGHT_CONST, window=DEFAULT_WINDOW):
    """fuse_depth with the previous output depth as one more input at the same pixel (weight tmp_weight).
    Returns dict(depth, index, ambiguous, wview) with wview = sum of the views' weights at the crossing."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    td = np.ascontiguousarray(tmp_depth, np.float32)
    tw = np.ascontiguousarray(tmp_weight, np.float32)
    shape = (target.height, target.width)
    out_d = np.empty(shape, np.float64)
    out_i = np.empty(shape, np.int32)
    out_a = np.empty(shape, np.uint8)
    out_w = np.empty(shape, np.float64)
    rc = lib.orc_fuse_depth_temporal(_cams(in_cams), _ptr(depths), len(in_cams), ctypes.byref(_cam(target)),
                                     int(num_samples), float(np.float32(z_near)), float(np.float32(z_far)),
                                     float(np.float32(mu)), float(weight_const), int(window), _ptr(td), _ptr(tw),
                                     _ptr(out_d), _ptr(out_i), _ptr(out_a), _ptr(out_w))
    if rc != 0:
        raise ValueError("orc_fuse_depth_temporal rejected its arguments")
    return {"depth": out_d, "index": out_i, "ambiguous": out_a, "wview": out_w}


def fuse_depth_grad(in_cams, depths, target, num_samples, z_near, z_far, mu, grad_fused,
                    weight_const=DEFAULT_WEIGHT_CONST, window=DEFAULT_WINDOW):
    """Adjoint of fuse_depth (normalize off): d(sum grad_fused * D) / d depths, float64 [N, H, W]."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    g = np.ascontiguousarray(grad_fused, np.float64)
    out = np.zeros(depths.shape, np.float64)
    rc = lib.orc_fuse_depth_grad(_cams(in_cams), _ptr(depths), len(in_cams), ctypes.byref(_cam(target)),
                                 int(num_samples), float(np.float32(z_near)), float(np.float32(z_far)),
                                 float(np.float32(mu)), float(weight_const), int(window), _ptr(g), _ptr(out))
    if rc != 0:
        raise ValueError("orc_fuse_depth_grad rejected its arguments")
    return out


def forward_splat(in_cams, depths, rgba_u32, target, footprint=True, max_half_width=2.0, mu_guide=0.04,
                  fused=None, count_fp64=False, guide_reject=False):
    """Per-view z-buffered forward render into the target.  guide_reject: candidates with
    z < float32(fused) - mu_guide (FP32) take no part in the depth test (needs `fused`).

    Returns dict(winner int32 [N, Ht, Wt] (-1 none), warped_rgba uint32, warped_depth float32,
    alpha uint8, guided uint8, guided_ambiguous uint8, fp64_mismatch int)."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    rgba_u32 = np.ascontiguousarray(rgba_u32, np.uint32)
    N = len(in_cams)
    shape = (N, target.height, target.width)
    win = np.empty(shape, np.int32)
    wr = np.empty(shape, np.uint32)
    wd = np.empty(shape, np.float32)
    al = np.empty(shape, np.uint8)
    gu = np.zeros(shape, np.uint8)
    ga = np.zeros(shape, np.uint8)
    fz = None if fused is None else np.ascontiguousarray(fused, np.float64)
    mism = ctypes.c_int64(0)
    rc = lib.orc_forward_splat(_cams(in_cams), _ptr(depths), _ptr(rgba_u32), N, ctypes.byref(_cam(target)),
                               int(bool(footprint)), ctypes.c_float(max_half_width), ctypes.c_float(mu_guide),
                               int(bool(guide_reject)), _ptr(fz), _ptr(win), _ptr(wr), _ptr(wd), _ptr(al), _ptr(gu), _ptr(ga),
                               ctypes.addressof(mism) if count_fp64 else None)
    if rc != 0:
        raise ValueError("orc_forward_splat rejected its arguments")
    return {"winner": win, "warped_rgba": wr, "warped_depth": wd, "alpha": al, "guided": gu,
            "guided_ambiguous": ga, "fp64_mismatch": int(mism.value)}


def soft_splat(in_cams, depths, colors, target, max_half_width=2.0, mu_band=0.04):
    """Differentiable colour splat (footprint mode).  colors float [N, H, W, 4] in [0, 1].

    Returns dict(winner int32, color float64 [N, Ht, Wt, 4], depth float32, wsum float64, alpha uint8)."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    colors = np.ascontiguousarray(colors, np.float64)
    N = len(in_cams)
    shape = (N, target.height, target.width)
    win = np.empty(shape, np.int32)
    col = np.empty(shape + (4,), np.float64)
    dep = np.empty(shape, np.float32)
    wsum = np.empty(shape, np.float64)
    al = np.empty(shape, np.uint8)
    rc = lib.orc_soft_splat(_cams(in_cams), _ptr(depths), _ptr(colors), N, ctypes.byref(_cam(target)),
                            ctypes.c_float(max_half_width), ctypes.c_float(mu_band), _ptr(win), _ptr(col), _ptr(dep),
                            _ptr(wsum), _ptr(al))
    if rc != 0:
        raise ValueError("orc_soft_splat rejected its arguments")
    return {"winner": win, "color": col, "depth": dep, "wsum": wsum, "alpha": al}


def soft_splat_grad(in_cams, depths, colors, target, grad_color, grad_depth=None, max_half_width=2.0, mu_band=0.04):
    """Adjoint of soft_splat: (grad w.r.t. depths float64 [N, H, W], w.r.t. colors float64 [N, H, W, 4])."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    colors = np.ascontiguousarray(colors, np.float64)
    gc = np.ascontiguousarray(grad_color, np.float64)
    gd = None if grad_depth is None else np.ascontiguousarray(grad_depth, np.float64)
    out_d = np.zeros(depths.shape, np.float64)
    out_c = np.zeros(colors.shape, np.float64)
    rc = lib.orc_soft_splat_grad(_cams(in_cams), _ptr(depths), _ptr(colors), len(in_cams), ctypes.byref(_cam(target)),
                                 ctypes.c_float(max_half_width), ctypes.c_float(mu_band), _ptr(gc), _ptr(gd),
                                 _ptr(out_d), _ptr(out_c))
    if rc != 0:
        raise ValueError("orc_soft_splat_grad rejected its arguments")
    return out_d, out_c


def splat_bruteforce(in_cams, depths, target, footprint=True, max_half_width=2.0):
    """Target-major enumeration of every (source, covered target) candidate; winner map only."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    N = len(in_cams)
    win = np.empty((N, target.height, target.width), np.int32)
    lib.orc_splat_bruteforce(_cams(in_cams), _ptr(depths), N, ctypes.byref(_cam(target)), int(bool(footprint)),
                             ctypes.c_float(max_half_width), _ptr(win))
    return win


def gauss_splat(in_cams, depths, rgba_u32, target, scale_px=0.5, max_radius=8, pixels=None):
    """Pixel-sized Gaussians, alpha-composited per view (Sec. 3.1, Supplement A.3).
    pixels: flat target indices (j * Wt + i) or None for the whole target.

    Returns dict(color float64 [N, P, 4] (premultiplied rgb, opacity), depth float64 [N, P],
    ambiguous uint8 [N, P]) with P = Ht * Wt (reshaped to [N, Ht, Wt(, 4)]) when pixels is None."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    rgba_u32 = np.ascontiguousarray(rgba_u32, np.uint32)
    N = len(in_cams)
    px = None if pixels is None else np.ascontiguousarray(pixels, np.int32)
    P = target.width * target.height if px is None else len(px)
    col = np.empty((N, P, 4), np.float64)
    dep = np.empty((N, P), np.float64)
    amb = np.zeros((N, P), np.uint8)
    rc = lib.orc_gauss_splat(_cams(in_cams), _ptr(depths), _ptr(rgba_u32), N, ctypes.byref(_cam(target)),
                             ctypes.c_float(scale_px), int(max_radius), _ptr(px), P, _ptr(col), _ptr(dep),
                             _ptr(amb))
    if rc != 0:
        raise ValueError("orc_gauss_splat rejected its arguments")
    if px is None:
        col = col.reshape(N, target.height, target.width, 4)
        dep = dep.reshape(N, target.height, target.width)
        amb = amb.reshape(N, target.height, target.width)
    return {"color": col, "depth": dep, "ambiguous": amb}


def blend_features(in_cams, target, warped_rgba, warped_depth, alpha, fused):
    """The (9K + 1) x Ht x Wt input of the blending network (Sec. 3.3 and the supplement's
    input list), FP64.  warped_rgba uint32 [K, Ht, Wt], warped_depth float32, alpha uint8,
    fused float32 [Ht, Wt]."""
    lib = _load()
    K = len(in_cams)
    wr = np.ascontiguousarray(warped_rgba, np.uint32)
    wd = np.ascontiguousarray(warped_depth, np.float32)
    al = np.ascontiguousarray(alpha, np.uint8)
    fz = np.ascontiguousarray(fused, np.float32)
    out = np.empty((9 * K + 1, target.height, target.width), np.float64)
    rc = lib.orc_blend_features(_cams(in_cams), K, ctypes.byref(_cam(target)), _ptr(wr), _ptr(wd), _ptr(al),
                                _ptr(fz), _ptr(out))
    if rc != 0:
        raise ValueError("orc_blend_features rejected its arguments")
    return out


def blend(warped_rgba, alpha, warped_depth, fused, w, w_bg, i_bg):
    """Eqs. 4-5 and L_Depth.  w float [K, H, W], w_bg [H, W], i_bg [3, H, W].
    Returns (image float64 [3, H, W], L_Depth)."""
    lib = _load()
    wr = np.ascontiguousarray(warped_rgba, np.uint32)
    K, H, W = wr.shape
    out = np.empty((3, H, W), np.float64)
    L = ctypes.c_double(0.0)
    rc = lib.orc_blend(K, W, H, _ptr(wr), _ptr(np.ascontiguousarray(alpha, np.uint8)),
                       _ptr(np.ascontiguousarray(warped_depth, np.float32)),
                       _ptr(np.ascontiguousarray(fused, np.float32)), _ptr(np.ascontiguousarray(w, np.float64)),
                       _ptr(np.ascontiguousarray(w_bg, np.float64)), _ptr(np.ascontiguousarray(i_bg, np.float64)),
                       _ptr(out), ctypes.addressof(L))
    if rc != 0:
        raise ValueError("orc_blend rejected its arguments")
    return out, L.value


def weight_f32(depth, u, v, mu, weight_const=0.001, window=7):
    """Supplement A.1's confidence weight as the sphere-tracing path evaluates it (FP32)."""
    lib = _load()
    d = np.ascontiguousarray(depth, np.float32)
    H, W = d.shape
    return float(lib.orc_weight_f32(_ptr(d), H, W, int(u), int(v), ctypes.c_float(mu), ctypes.c_float(weight_const),
                                    int(window), ctypes.c_float(1.0 / (window * window))))


def fuse_depth_sphere(in_cams, depths, target, z_near, z_far, mu, weight_const=0.001, window=7, max_steps=1024,
                      min_frac=0.0625):
    """Supplement A.1's raymarch (0.8 s steps, three bisections), FP32 as the kernel takes it.

    Returns dict(depth float32 [Ht, Wt] (0: no crossing), evals int32 [Ht, Wt])."""
    lib = _load()
    depths = np.ascontiguousarray(depths, np.float32)
    out = np.empty((target.height, target.width), np.float32)
    ev = np.empty((target.height, target.width), np.int32)
    rc = lib.orc_fuse_depth_sphere(_cams(in_cams), _ptr(depths), len(in_cams), ctypes.byref(_cam(target)),
                                   float(z_near), float(z_far), float(mu), float(weight_const), int(window),
                                   int(max_steps), float(min_frac), _ptr(out), _ptr(ev))
    if rc != 0:
        raise ValueError("orc_fuse_depth_sphere rejected its arguments")
    return {"depth": out, "evals": ev}


def uniform_blend_loss(color, alpha, warped_depth, fused, gt, w_l1=0.8, w_depth=0.1):
    """Sec. 3.3's training loss on the uniform blend of the views (Eq. 4 with every
    w_k = 1, the denominator read as the sum over the views), written out in FP64:
      A(p) = sum_k a_k(p),  B(p) = sum_k a_k I_k(p) / A(p)   (pixels with A > 0, n of them)
      L1 = sum_{A>0} sum_rgb |B - GT| / (3 n)
      Dbar(p) = sum_k a_k D_k(p) / A(p) (0 where A = 0),  v(p) = [A > 0 and F(p) > 0]
      L_Depth = sum_p v |F - Dbar| / (K H W)        (the printed 1/(HWK))
      L = w_l1 L1 + w_depth L_Depth
    color [K, H, W, 3 or 4] (RGB used), alpha [K, H, W] (0/1), warped_depth [K, H, W],
    fused [H, W], gt [H, W, 3].  Returns (L, L1, L_Depth, grads) with grads the derivatives
    d L / d I_k (= a_k g_rgb), d L / d D_k (= a_k g_d) and d L / d F, as per-pixel
    g_rgb [H, W, 3], g_d [H, W] and g_F [H, W] (|x|' = sign(x), 0 at 0)."""
    I = np.asarray(color, np.float64)[..., :3]
    a = np.asarray(alpha, np.float64)
    D = np.asarray(warped_depth, np.float64)
    F = np.asarray(fused, np.float64)
    G = np.asarray(gt, np.float64)
    K, H, W = a.shape
    A = a.sum(0)
    cov = A > 0
    inv = np.where(cov, 1.0 / np.maximum(A, 1.0), 0.0)
    B = (a[..., None] * I).sum(0) * inv[..., None]
    n = max(int(cov.sum()), 1)
    L1 = np.abs(B - G)[cov].sum() / (3.0 * n)
    Dbar = (a * D).sum(0) * inv
    v = cov & (F > 0)
    LD = np.abs(F - Dbar)[v].sum() / (K * H * W)
    g_rgb = w_l1 * np.sign(B - G) / (3.0 * n) * inv[..., None] * cov[..., None]
    sd = np.sign(F - Dbar) * v
    g_d = -w_depth * sd / (K * H * W) * inv
    g_F = w_depth * sd / (K * H * W)
    return w_l1 * L1 + w_depth * LD, L1, LD, {"rgb": g_rgb, "depth": g_d, "fused": g_F}
