"""Pins for the oracle's differentiable colour splat and its adjoint.

* identity camera: every target pixel is covered by its own source pixel only,
  so the colour is copied, d colour / d colour is the identity and the warped
  depth's gradient reaches the source depth with slope dz/dd = 1;
* winner, warped depth and alpha equal the hard z-buffer splat's;
* colour gradients are exact (the colour is linear in the source colours);
* depth gradients against central finite differences, redrawing samples whose
  two step sizes disagree (a pixel entering or leaving a footprint or the
  front band inside the step).
"""
import numpy as np
import pytest


def _colors(rgb):
    return np.ascontiguousarray(rgb, np.float64) / 255.0


def test_identity_camera(oracle_mod, synth_mod):
    from synth import configs, render
    from synth.configs import arc_cameras
    cam = arc_cameras(40, 30, [9.0])[0]
    rgb, d = render(configs.plain_320x240().scene(0), cam, noise_sigma=0.002, noise_seed=4)
    col = _colors(rgb)[None]
    r = oracle_mod.soft_splat([cam], d[None], col, cam)
    np.testing.assert_allclose(r["color"][0, ..., :3], col[0, ..., :3], atol=1e-12)
    rng = np.random.default_rng(0)
    Gc = rng.standard_normal((1, 30, 40, 4))
    Gd = rng.standard_normal((1, 30, 40))
    gd, gc = oracle_mod.soft_splat_grad([cam], d[None], col, cam, Gc, Gd)
    np.testing.assert_allclose(gc[..., :3], Gc[..., :3], atol=1e-9)
    assert np.abs(gc[..., 3]).max() == 0.0
    np.testing.assert_allclose(gd, Gd, rtol=1e-5, atol=1e-4)


def test_matches_hard_splat(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(48, 32, 3, 16)
    rgb, d = w.render_inputs(0)
    s = oracle_mod.soft_splat(w.inputs, d, _colors(rgb), w.targets[0])
    h = oracle_mod.forward_splat(w.inputs, d, np.ascontiguousarray(rgb).view(np.uint32)[..., 0], w.targets[0])
    assert np.array_equal(s["winner"], h["winner"])
    assert np.array_equal(s["alpha"], h["alpha"])
    assert np.array_equal(s["depth"].view(np.uint32), h["warped_depth"].view(np.uint32))
    covered = s["alpha"] == 1
    assert (s["wsum"][covered] > 0).all()
    assert (s["color"][covered][:, :3] >= 0).all() and (s["color"][covered][:, :3] <= 1).all()


def _loss(oracle_mod, w, d, col, Gc, Gd):
    r = oracle_mod.soft_splat(w.inputs, d, col, w.targets[0])
    return float((r["color"] * Gc).sum() + (r["depth"].astype(np.float64) * Gd).sum()), r["winner"]


def test_finite_differences(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(36, 28, 2, 16)
    t = w.targets[0]
    t.fx, t.fy = t.fx * 1.7, t.fy * 1.7        # magnified: footprints wider than a pixel
    rgb, d = w.render_inputs(0)
    col = _colors(rgb)
    rng = np.random.default_rng(7)
    Gc = rng.standard_normal((2, 28, 36, 4))
    Gd = 0.1 * rng.standard_normal((2, 28, 36))
    gd, gc = oracle_mod.soft_splat_grad(w.inputs, d, col, t, Gc, Gd)
    _, win0 = _loss(oracle_mod, w, d, col, Gc, Gd)
    # colour: linear, so the central difference is exact up to rounding
    for k, v, u, ch in [(0, 5, 7, 0), (1, 20, 30, 2), (0, 14, 14, 1)]:
        cp, cm = col.copy(), col.copy()
        cp[k, v, u, ch] += 1e-3
        cm[k, v, u, ch] -= 1e-3
        fd = (_loss(oracle_mod, w, d, cp, Gc, Gd)[0] - _loss(oracle_mod, w, d, cm, Gc, Gd)[0]) / 2e-3
        assert fd == pytest.approx(gc[k, v, u, ch], rel=1e-7, abs=1e-9)
    scale = np.abs(gd).max()
    checked = 0
    for k, v, u in np.argwhere(np.abs(gd) > 1e-3 * scale)[rng.choice((np.abs(gd) > 1e-3 * scale).sum(), 40,
                                                                     replace=False)]:
        fd = []
        for h in (1e-3, 5e-4):
            dp, dm = d.copy(), d.copy()
            dp[k, v, u] += np.float32(h)
            dm[k, v, u] -= np.float32(h)
            lp, wp = _loss(oracle_mod, w, dp, col, Gc, Gd)
            lm, wm = _loss(oracle_mod, w, dm, col, Gc, Gd)
            if not (np.array_equal(wp, win0) and np.array_equal(wm, win0)):
                fd = None
                break
            fd.append((lp - lm) / (float(dp[k, v, u]) - float(dm[k, v, u])))
        if fd is None or abs(fd[0] - fd[1]) > 1e-3 * scale:
            continue
        checked += 1
        assert abs(fd[1] - gd[k, v, u]) <= 1e-2 * scale, (k, v, u, fd, gd[k, v, u])
    assert checked >= 20
