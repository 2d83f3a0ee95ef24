"""Host-side checks of the C ABI: the library loads, exports every symbol that
include/*.h declares, and rejects bad arguments before enqueuing anything.
No call here reaches a kernel, so none needs a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_18932_gb300 import build as b
    b.build()
    from paper_2505_18932_gb300 import gvs
    return gvs.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"GVS_API\s+[\w\s\*]*?\b(gvs_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ["gvs_refine_depth", "gvs_fuse_depth", "gvs_forward_splat", "gvs_fuse_workspace_bytes",
              "gvs_splat_workspace_bytes", "gvs_last_error", "gvs_version", "gvs_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2505_18932_gb300 import gvs
    assert set(declared_symbols()) <= set(gvs.API)


def _cam(gvs, W=64, H=48):
    from synth import camera_at
    return gvs.camera_struct(camera_at(W, H, (0.0, 0.0, 0.0)))


FAKE = 0x10000  # a 256-byte aligned stand-in address; never dereferenced on these paths


def test_fuse_rejects_bad_arguments(lib):
    from paper_2505_18932_gb300 import gvs
    cams = (gvs.GvsCamera * 2)(_cam(gvs), _cam(gvs))
    tgt = _cam(gvs)
    good = dict(num_samples=64, z_near=0.5, z_far=5.0, mu=0.05, weight_const=0.001, window=7, normalize=0,
                depth_dtype=0, map_dtype=0)
    ws = lib.gvs_fuse_workspace_bytes(2, 64, 48)
    assert ws >= 2 * 64 * 48 * 8 and ws % 256 == 0

    def call(params=good, cams=cams, n=2, target=tgt, fused=FAKE, wsp=FAKE, wsb=ws, depths=FAKE):
        p = gvs.GvsFuseParams(**params)
        return lib.gvs_fuse_depth(cams, depths, n, ctypes.byref(target) if target is not None else None,
                                  ctypes.byref(p), fused, None, wsp, wsb, None)

    for bad in [dict(num_samples=1), dict(z_near=0.0), dict(z_near=5.0), dict(mu=0.0), dict(mu=float("nan")),
                dict(window=6), dict(window=17), dict(normalize=2), dict(weight_const=-1.0),
                dict(num_samples=40000)]:
        assert call(params={**good, **bad}) == 1, bad
        assert lib.gvs_last_error()
    assert call(n=33) == 1
    assert call(n=-1) == 1
    assert call(params={**good, "depth_dtype": 2}) == 2     # bf16 depth is not a storage this path offers
    assert call(params={**good, "map_dtype": 7}) == 2
    assert call(fused=None) == 1
    assert call(fused=FAKE + 4) == 1           # misaligned
    assert call(depths=None) == 1
    assert call(wsb=ws - 1) == 3                # workspace too small
    assert call(wsp=FAKE + 16) == 3             # workspace misaligned
    bad_cam = _cam(gvs)
    bad_cam.fx = -1.0
    assert call(target=bad_cam) == 1
    odd = (gvs.GvsCamera * 2)(_cam(gvs), _cam(gvs, 32, 48))   # different input sizes
    assert call(cams=odd) == 1
    nan_cam = (gvs.GvsCamera * 2)(_cam(gvs), _cam(gvs))
    nan_cam[1].R[4] = float("nan")
    assert call(cams=nan_cam) == 1


def test_splat_rejects_bad_arguments(lib):
    from paper_2505_18932_gb300 import gvs
    cams = (gvs.GvsCamera * 1)(_cam(gvs))
    tgt = _cam(gvs)
    ws = lib.gvs_splat_workspace_bytes(1, 64, 48)
    assert ws == 64 * 48 * 8

    def call(fp=1, mhw=2.0, mug=0.04, fused=FAKE, guided=FAKE, winner=FAKE, wsb=ws):
        p = gvs.GvsSplatParams(fp, mhw, mug)
        return lib.gvs_forward_splat(cams, FAKE, FAKE, 1, ctypes.byref(tgt), ctypes.byref(p), fused, winner,
                                     None, None, None, guided, FAKE, wsb, None)

    assert call(fp=2) == 1
    p_bad = gvs.GvsSplatParams(1, 2.0, 0.04, 2)
    assert lib.gvs_forward_splat(cams, FAKE, FAKE, 1, ctypes.byref(tgt), ctypes.byref(p_bad), FAKE, FAKE,
                                 None, None, None, FAKE, FAKE, ws, None) == 2
    assert call(mhw=0.25) == 1
    assert call(mug=-1.0) == 1
    assert call(fused=None) == 1       # guided mask without the fused depth
    assert call(winner=None) == 1
    assert call(winner=FAKE + 8) == 1
    assert call(wsb=ws - 8) == 3


def test_splat_guide_reject_arguments(lib):
    from paper_2505_18932_gb300 import gvs
    cams = (gvs.GvsCamera * 1)(_cam(gvs))
    tgt = _cam(gvs)
    ws = lib.gvs_splat_workspace_bytes(1, 64, 48)

    def call(rej, fused=FAKE, mug=0.04):
        p = gvs.GvsSplatParams(1, 2.0, mug, 0, rej)
        return lib.gvs_forward_splat(cams, FAKE, FAKE, 1, ctypes.byref(tgt), ctypes.byref(p), fused, FAKE,
                                     None, None, None, None, FAKE, ws, None)

    assert call(2) == 1
    assert call(1, fused=None) == 1     # rejection needs the fused depth
    assert call(1, mug=float("nan")) == 1


def test_gauss_splat_rejects_bad_arguments(lib):
    from paper_2505_18932_gb300 import gvs
    cams = (gvs.GvsCamera * 1)(_cam(gvs))
    tgt = _cam(gvs)
    ws = lib.gvs_gauss_splat_workspace_bytes(64, 48, 64, 48, 8)
    # records, 4 x 3 tile counters and offsets, at most 9 tile entries per source pixel
    assert ws >= 64 * 48 * 32 + 64 * 48 * 9 * 8
    assert lib.gvs_gauss_splat_workspace_bytes(64, 48, 64, 48, 0) == 0
    assert lib.gvs_gauss_splat_workspace_bytes(64, 48, 64, 48, 33) == 0

    def call(scale=0.5, rmax=8, dt=0, color=FAKE, depth=FAKE, wsb=ws, params=True):
        p = gvs.GvsGaussParams(scale, rmax, dt)
        return lib.gvs_gauss_splat(cams, FAKE, FAKE, 1, ctypes.byref(tgt), ctypes.byref(p) if params else None,
                                   color, depth, FAKE, wsb, None)

    assert call(params=False) == 1
    assert call(scale=0.0) == 1
    assert call(scale=float("inf")) == 1
    assert call(rmax=0) == 1
    assert call(rmax=33) == 1
    assert call(dt=2) == 2
    assert call(color=None) == 1
    assert call(depth=FAKE + 4) == 1
    assert call(wsb=ws - 256) == 3


def test_refine_rejects_bad_arguments(lib):
    from paper_2505_18932_gb300 import gvs

    def call(tau=0.03, n=2, W=64, H=48, rgba=FAKE, depth=FAKE, state=FAKE):
        p = gvs.GvsRefineParams(tau)
        return lib.gvs_refine_depth(rgba, FAKE, depth, state, None, n, W, H, ctypes.byref(p), None)

    assert lib.gvs_refine_depth(FAKE, FAKE, FAKE, FAKE, None, 1, 4, 4, ctypes.byref(gvs.GvsRefineParams(0.03, 2)),
                                None) == 2
    assert call(tau=-0.1) == 1
    assert call(tau=1.5) == 1
    assert call(tau=float("nan")) == 1
    assert call(n=33) == 1
    assert call(W=0) == 1
    assert call(H=20000) == 1
    assert call(rgba=None) == 1
    assert call(state=FAKE + 4) == 1
    assert call(n=0) == 0           # no views: nothing to do
    assert lib.gvs_refine_depth(FAKE, FAKE, FAKE, FAKE, None, 1, 4, 4, None, None) == 1


def test_blend_loss_rejects_bad_arguments(lib):
    """gvs_uniform_blend_loss and its gradient stage check sizes, outputs, alignment and the
    workspace on the host, before anything is enqueued."""
    W, H = 64, 48
    ws = lib.gvs_uniform_blend_loss_workspace_bytes(W, H)
    assert ws >= W * H * 4
    assert lib.gvs_uniform_blend_loss_workspace_bytes(0, H) == 0

    def loss(n=2, W=W, H=H, color=FAKE, w_l1=0.8, lossp=FAKE, gp=FAKE, wsp=FAKE, wsb=ws):
        return lib.gvs_uniform_blend_loss(n, W, H, color, FAKE, FAKE, FAKE, FAKE, w_l1, 0.1, lossp, gp, None,
                                          wsp, wsb, None)

    assert loss(n=0) == 1
    assert loss(n=33) == 1
    assert loss(W=0) == 1
    assert loss(w_l1=-1.0) == 1
    assert loss(w_l1=float("inf")) == 1
    assert loss(color=None) == 1
    assert loss(color=FAKE + 4) == 1
    assert loss(lossp=FAKE + 4) == 1
    assert loss(gp=FAKE + 4) == 1
    assert loss(wsp=None) == 3
    assert loss(wsb=ws - 1) == 3
    assert loss(wsp=FAKE + 16) == 3

    def grad(W=W, H=H, gl=FAKE, gp=FAKE, gf=FAKE, wsp=FAKE, wsb=ws):
        return lib.gvs_uniform_blend_loss_grad(W, H, gl, gp, gf, wsp, wsb, None)

    assert grad(W=0) == 1
    assert grad(H=20000) == 1
    assert grad(gp=None, gf=None) == 1
    assert grad(gp=FAKE + 4) == 1
    assert grad(gf=FAKE + 2) == 1
    assert grad(gl=FAKE + 2) == 1
    assert grad(wsp=None) == 3
    assert grad(wsb=ws - 256) == 3
    assert grad(wsp=FAKE + 16) == 3


def test_status_strings(lib):
    for s in range(6):
        assert lib.gvs_status_string(s)
    assert lib.gvs_version().startswith(b"gvs")


def test_binding_refuses_cpu_tensors():
    import torch
    from paper_2505_18932_gb300 import gvs
    with pytest.raises(ValueError):
        gvs._ptr(torch.zeros(4))


def test_select_views_host_only(lib):
    """K-closest selection is host code: checked here without a GPU against distances
    computed independently."""
    import numpy as np
    from paper_2505_18932_gb300 import gvs
    from synth import camera_at, look_at
    rng = np.random.default_rng(0)
    centres = rng.uniform(-1, 1, (9, 3))
    cams = [look_at(64, 48, c, (0.0, 0.0, 3.0)) if i % 2 else camera_at(64, 48, c) for i, c in enumerate(centres)]
    tgt = camera_at(64, 48, (0.1, -0.2, 0.05))
    for k in (1, 4, 9):
        got = gvs.select_views(cams, tgt, k)
        d = np.linalg.norm(centres - np.array([0.1, -0.2, 0.05]), axis=1)
        assert got == list(np.argsort(d, kind="stable")[:k])
    twins = [camera_at(64, 48, (1.0, 0, 0)), camera_at(64, 48, (-1.0, 0, 0)), camera_at(64, 48, (0, 0.5, 0))]
    assert gvs.select_views(twins, camera_at(64, 48, (0, 0, 0)), 3) == [2, 0, 1]   # tie -> lower index
    with pytest.raises(gvs.GvsError):
        gvs.select_views(twins, camera_at(64, 48, (0, 0, 0)), 4)


def test_normal_build_checks_no_bounds(lib):
    """Without GVS_BOUNDS_CHECK the debug accessor is a constant 0 (no CUDA call)."""
    assert lib.gvs_debug_bounds_error() == 0
