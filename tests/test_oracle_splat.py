"""Pins for the oracle's per-view forward splat (Sec. 3.1, Supplement A.3).

Closed forms (identity camera, integer disparity of a fronto-parallel plane),
brute-force enumeration on tiny images, agreement of the FP32 address contract
with FP64 geometry, and the depth test keeping the front surface.
"""
import numpy as np
import pytest


def _u32(rgba):
    return np.ascontiguousarray(rgba).view(np.uint32)[..., 0]


@pytest.mark.parametrize("deg", [0.0, 11.0])
def test_identity_camera_point_mode(oracle_mod, synth_mod, deg):
    from synth import configs
    from synth.configs import arc_cameras
    cam = arc_cameras(48, 32, [deg])[0]
    w = configs.plain_320x240()
    from synth import render
    rgb, d = render(w.scene(0), cam, noise_sigma=0.002, noise_seed=5)
    r = oracle_mod.forward_splat([cam], d[None], _u32(rgb)[None], cam, footprint=False)
    idx = np.arange(48 * 32).reshape(32, 48)
    assert np.array_equal(r["winner"][0], idx)
    assert np.array_equal(r["warped_rgba"][0], _u32(rgb))
    np.testing.assert_allclose(r["warped_depth"][0], d, rtol=1e-6)
    assert r["alpha"].min() == 1


@pytest.mark.parametrize("footprint", [False, True])
def test_integer_disparity_plane(oracle_mod, synth_mod, footprint):
    """Source camera shifted by +tx along x, plane at depth d with f*tx/d = 5 px:
    target pixel i sees source pixel i - 5 on the same row."""
    from synth import camera_at
    W, H = 40, 24
    tgt = camera_at(W, H, (0.0, 0.0, 0.0))
    d = 2.0
    tx = 5.0 * d / tgt.fx
    src = camera_at(W, H, (tx, 0.0, 0.0))
    dep = np.full((1, H, W), d, np.float32)
    rgb = np.arange(W * H, dtype=np.uint32).reshape(1, H, W)
    r = oracle_mod.forward_splat([src], dep, rgb, tgt, footprint=footprint)
    win = r["winner"][0]
    jj, ii = np.mgrid[0:H, 0:W]
    exp = np.where(ii >= 5, jj * W + (ii - 5), -1)
    # footprint mode: half-width 0.5 covers exactly one pixel unless x sits on a
    # half-integer; with integer disparity x is an integer
    assert np.array_equal(win, exp)
    # the colour of source pixel n is n, so the warped colour is the winner index
    assert np.array_equal(r["warped_rgba"][0][ii >= 5], exp[ii >= 5].astype(np.uint32))


def test_bruteforce_tiny(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(16, 16, 3, 8)
    rgb, d = w.render_inputs(0)
    d[1, 3:6, 4:9] = 0.0   # some invalid source pixels
    for fp in (False, True):
        r = oracle_mod.forward_splat(w.inputs, d, _u32(rgb), w.targets[0], footprint=fp)
        bf = oracle_mod.splat_bruteforce(w.inputs, d, w.targets[0], footprint=fp)
        assert np.array_equal(r["winner"], bf)
        assert (r["winner"] >= 0).mean() > 0.5


def test_contract_agrees_with_fp64_geometry(oracle_mod, synth_mod):
    from synth import configs
    w = configs.plain_320x240()
    rgb, d = w.render_inputs(0)
    r = oracle_mod.forward_splat(w.inputs, d, _u32(rgb), w.targets[0], count_fp64=True)
    n = r["winner"].size
    assert r["fp64_mismatch"] < 1e-3 * n


def test_depth_test_keeps_front_surface(oracle_mod, synth_mod):
    """Warped depth must match the target's analytic depth where a sphere occludes
    the background; an argmax instead of argmin would show the background."""
    from synth import configs, render
    w = configs.plain_320x240()
    sc = w.scene(0)
    rgb, d = w.render_inputs(0)
    _, gt = render(sc, w.targets[0])
    r = oracle_mod.forward_splat(w.inputs, d, _u32(rgb), w.targets[0])
    gy, gx = np.gradient(gt.astype(np.float64))
    smooth = np.abs(gx) + np.abs(gy) < 0.01 * gt
    for k in range(len(w.inputs)):
        m = (r["alpha"][k] == 1) & smooth
        err = np.abs(r["warped_depth"][k][m] - gt[m]) / gt[m]
        assert np.median(err) < 5e-3


def test_guided_mask_definition(oracle_mod, synth_mod):
    """With the fused depth equal to each view's own warped depth the guided mask equals alpha;
    shifted by more than mu_guide it is empty."""
    from synth import configs
    w = configs.tiny(32, 24, 2, 16)
    rgb, d = w.render_inputs(0)
    r0 = oracle_mod.forward_splat(w.inputs[:1], d[:1], _u32(rgb)[:1], w.targets[0])
    fused = r0["warped_depth"][0].astype(np.float64)
    r = oracle_mod.forward_splat(w.inputs[:1], d[:1], _u32(rgb)[:1], w.targets[0], mu_guide=0.04, fused=fused)
    assert np.array_equal(r["guided"][0], r["alpha"][0])
    r = oracle_mod.forward_splat(w.inputs[:1], d[:1], _u32(rgb)[:1], w.targets[0], mu_guide=0.04,
                                 fused=fused + 0.05)
    assert r["guided"].max() == 0


def _occluder_case():
    """Source camera shifted along x; a background plane at depth 2 and a square
    occluder at depth 1 in the source view, so the occluder covers background
    pixels in the target (parallax of 10 px against 5 px)."""
    from synth import camera_at
    W, H = 48, 32
    tgt = camera_at(W, H, (0.0, 0.0, 0.0))
    src = camera_at(W, H, (10.0 / tgt.fx, 0.0, 0.0))
    dep = np.full((1, H, W), 2.0, np.float32)
    dep[0, 8:20, 14:30] = 1.0
    rgb = np.arange(W * H, dtype=np.uint32).reshape(1, H, W)
    return src, tgt, dep, rgb


def test_guide_reject_drops_surfaces_in_front(oracle_mod, synth_mod):
    """With the fused depth on the background plane everywhere, rejecting candidates in
    front of fused - mu equals splatting a source whose occluder pixels are invalid; a
    fused depth of 0 (no crossing) rejects nothing; one far behind everything rejects all."""
    src, tgt, dep, rgb = _occluder_case()
    H, W = dep.shape[1:]
    plane = np.full((H, W), 2.0)
    r = oracle_mod.forward_splat([src], dep, rgb, tgt, fused=plane, mu_guide=0.04, guide_reject=True)
    cut = dep.copy()
    cut[dep < 1.5] = 0.0
    ref = oracle_mod.forward_splat([src], cut, rgb, tgt)
    assert np.array_equal(r["winner"], ref["winner"])
    plain = oracle_mod.forward_splat([src], dep, rgb, tgt)
    assert not np.array_equal(plain["winner"], ref["winner"])   # the occluder did win somewhere
    r0 = oracle_mod.forward_splat([src], dep, rgb, tgt, fused=np.zeros((H, W)), mu_guide=0.04, guide_reject=True)
    assert np.array_equal(r0["winner"], plain["winner"])
    far = oracle_mod.forward_splat([src], dep, rgb, tgt, fused=np.full((H, W), 50.0), mu_guide=0.04,
                                   guide_reject=True)
    assert far["winner"].max() == -1
    # mu: a fused depth 0.5 in front of the plane still keeps the plane (z >= fused - mu) only if mu >= 0.5
    near = np.full((H, W), 2.5)
    kept = oracle_mod.forward_splat([src], cut, rgb, tgt, fused=near, mu_guide=0.5, guide_reject=True)
    dropped = oracle_mod.forward_splat([src], cut, rgb, tgt, fused=near, mu_guide=0.49, guide_reject=True)
    assert np.array_equal(kept["winner"], ref["winner"]) and dropped["winner"].max() == -1
