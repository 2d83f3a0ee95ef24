"""Pins for the oracle's sphere-tracing raymarch (Supplement A.1: 0.8 s steps
until s changes sign, three bisection steps), taken in FP32 as the kernel
takes it.

Closed forms: a fronto-parallel plane is found within the final bracket
(|D - d| <= 0.8 mu min_frac / 16 plus rounding); with nothing observed the
march takes full-truncation steps, and with exactly representable steps the
number of evaluations is (z_far - z_near) / (0.8 mu) + 1; max_steps caps it.
The FP32 weight agrees with the FP64 weight of Supplement A.1, and on the
320x240 scene the traced depth agrees with the finely sampled uniform march.
"""
import numpy as np
import pytest


def _cam(W=48, H=32, x=0.0):
    from synth import Camera
    return Camera(W, H, 60.0, 60.0, (W - 1) / 2.0, (H - 1) / 2.0, np.eye(3), np.array([-x, 0.0, 0.0]))


@pytest.mark.parametrize("d", [1.0, 2.37, 3.9])
def test_plane_found_within_the_final_bracket(oracle_mod, synth_mod, d):
    cam = _cam()
    dep = np.full((1, 32, 48), d, np.float32)
    mu, mf = 0.04, 0.0625
    r = oracle_mod.fuse_depth_sphere([cam], dep, cam, 0.3, 8.0, mu, min_frac=mf)
    err = np.abs(r["depth"].astype(np.float64) - d)
    assert err.max() <= 0.8 * mu * mf / 16 + 4e-6 * d
    # free space first (steps of 0.8 mu), then the band: the count is bounded by the walk length
    assert r["evals"].min() >= 4 and r["evals"].max() <= (d - 0.3) / (0.8 * mu) + 1 / (0.8 * mf) + 8


def test_no_observation_full_truncation_steps(oracle_mod, synth_mod):
    """Nothing valid: W = 0 everywhere, steps of exactly 0.8 mu = 0.25 from 0.5 to 4.0."""
    cam = _cam()
    dep = np.zeros((1, 32, 48), np.float32)
    r = oracle_mod.fuse_depth_sphere([cam], dep, cam, 0.5, 4.0, 0.3125)
    assert np.all(r["depth"] == 0.0)
    assert np.all(r["evals"] == 15)
    r = oracle_mod.fuse_depth_sphere([cam], dep, cam, 0.5, 4.0, 0.3125, max_steps=5)
    assert np.all(r["evals"] == 5)


def test_weight_f32_matches_fp64(oracle_mod, synth_mod):
    rng = np.random.default_rng(4)
    d = (2.0 + 0.01 * rng.standard_normal((20, 24))).astype(np.float32)
    d[3, 4] = 0.0
    for (u, v) in [(0, 0), (5, 3), (23, 19), (10, 10), (4, 3)]:
        w64 = oracle_mod.weight(d, u, v, 0.04)
        w32 = oracle_mod.weight_f32(d, u, v, 0.04)
        assert w32 == pytest.approx(w64, rel=2e-6, abs=1e-30)


def test_agrees_with_fine_uniform_march(oracle_mod, synth_mod):
    """Both statements of Supplement A.1's fusion find the same surfaces."""
    from synth import configs
    w = configs.plain_320x240()
    _, d = w.render_inputs(0)
    tgt = w.targets[0]
    sph = oracle_mod.fuse_depth_sphere(w.inputs, d, tgt, w.z_near, w.z_far, w.mu)
    uni = oracle_mod.fuse_depth(w.inputs, d, tgt, 512, w.z_near, w.z_far, w.mu, normalize=True)
    both = (sph["depth"] > 0) & (uni["depth"] > 0)
    assert both.mean() > 0.5
    diff = np.abs(sph["depth"][both] - uni["depth"][both])
    assert np.median(diff) < 0.1 * w.mu and (diff < w.mu).mean() > 0.97


def test_plane_walk_worked_by_hand(oracle_mod, synth_mod):
    """Supplement A.1's rule walked by hand on a fronto-parallel plane at d = 2 seen by the
    target's own camera (flat depth: nu = 0, so every weight is 1 and s_n = clamp((d - z) / mu)),
    mu = 0.3125 (0.8 mu = 0.25), min_frac = 1/16, start 0.5:
      z = 0.5, 0.75, ..., 1.75   full steps of 0.25 while d - z >= mu (s_n = 1)   6 evaluations
      z = 1.75 -> 1.95           step 0.25 * 0.8   (s_n = 0.8)
      z = 1.95 -> 1.99           step 0.25 * 0.16  (s_n = 0.16)
      z = 1.99 -> 2.005625       step 0.25 / 16    (s_n = 0.032 < 1/16: the floor)
      z = 2.005625: s_n < 0 with weight on both sides -> bracket [1.99, 2.005625]   9 evaluations
      bisection: 1.9978125 (in front, keep upper), 2.00171875 (behind), 1.999765625 (in front)
      depth = midpoint of [1.999765625, 2.00171875] = 2.0007421875, 12 evaluations.
    The arithmetic is exact in real numbers; FP32 rounding moves no decision here."""
    cam = _cam()
    dep = np.full((1, 32, 48), 2.0, np.float32)
    r = oracle_mod.fuse_depth_sphere([cam], dep, cam, 0.5, 8.0, 0.3125, min_frac=0.0625)
    assert np.all(r["evals"] == 12)
    assert np.abs(r["depth"].astype(np.float64) - 2.0007421875).max() < 2e-6


def _fp64_plane_walk(d, z_near, z_far, mu, min_frac, max_steps=1024):
    """The same rule in FP64, for a plane at d seen by the target's own camera (weights 1)."""
    s_n = lambda z: None if (d - z) / mu < -1.0 else max(-1.0, min(1.0, (d - z) / mu))
    z, evals, prev = z_near, 0, None
    for _ in range(max_steps):
        if z > z_far:
            break
        s = s_n(z)
        evals += 1
        if prev is not None and prev[1] is not None and s is not None and prev[1] > 0.0 and s <= 0.0:
            lo, hi = prev[0], z
            for _ in range(3):
                m = 0.5 * (lo + hi)
                sm = s_n(m)
                evals += 1
                if sm is not None and sm > 0.0:
                    lo = m
                else:
                    hi = m
            return 0.5 * (lo + hi), evals, (lo, hi)
        prev = (z, s)
        z = z + 0.8 * mu * (1.0 if s is None else max(s, min_frac))
    return 0.0, evals, None


@pytest.mark.parametrize("d", [0.93, 1.7, 2.61, 4.4])
def test_plane_walk_matches_an_fp64_walk(oracle_mod, synth_mod, d):
    """The oracle's FP32 march against the rule taken in FP64 on a plane: the same number of
    evaluations, and the FP32 depth inside the FP64 walk's final bracket (up to FP32 rounding)."""
    cam = _cam()
    dep = np.full((1, 32, 48), d, np.float32)
    mu, mf = 0.04, 0.0625
    r = oracle_mod.fuse_depth_sphere([cam], dep, cam, 0.3, 8.0, mu, min_frac=mf)
    depth, evals, (lo, hi) = _fp64_plane_walk(float(np.float32(d)), 0.3, 8.0, mu, mf)
    assert np.all(r["evals"] == evals), (np.unique(r["evals"]), evals)
    got = r["depth"].astype(np.float64)
    assert np.all(got >= lo - 4e-7 * d) and np.all(got <= hi + 4e-7 * d)
