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
