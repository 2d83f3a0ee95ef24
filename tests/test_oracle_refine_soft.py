"""Pins for the paper's soft difference mask (Sec. 3.2, Eq. 1 and Eq. 2 as printed:
beta = 0.6, lambda_t = 0.7, quarter resolution, 3x3 max-pool, bilinear upsample).
Every expected value is worked out by hand for a constructed frame pair."""
import numpy as np
import pytest

BETA, LAM = 0.6, 0.7


def _frames(H=16, W=16, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 200, (1, H, W, 4), dtype=np.uint8)
    d = rng.uniform(1.0, 5.0, (1, H, W)).astype(np.float32)
    p = rng.uniform(1.0, 5.0, (1, H, W)).astype(np.float32)
    return a, d, p


def test_static_frame_keeps_forty_percent(oracle_mod):
    a, d, p = _frames()
    out, m = oracle_mod.refine_depth_soft(a, a, d, p)
    assert np.all(m == BETA)
    np.testing.assert_allclose(out, BETA * d.astype(np.float64) + (1 - BETA) * p.astype(np.float64), rtol=1e-15)


def test_uniform_change(oracle_mod):
    a, d, p = _frames()
    b = a.copy()
    b[..., 1] = np.clip(a[..., 1].astype(int) + 51, 0, 255).astype(np.uint8)   # +51 = 0.2 in green
    out, m = oracle_mod.refine_depth_soft(b, a, d, p)
    exp = min(0.2 / LAM + BETA, 1.0)
    np.testing.assert_allclose(m, exp, rtol=1e-14)
    b[..., 0] = 255 - a[..., 0]
    b[..., 0][np.abs(b[..., 0].astype(int) - a[..., 0]) < 200] = 0
    out, m = oracle_mod.refine_depth_soft(b, a, d, p)
    assert m.min() >= BETA and m.max() <= 1.0


def test_single_changed_pixel(oracle_mod):
    """One pixel changes by 255: its quarter cell averages 1/16, the 3x3 pool spreads
    0.6 + (1/16)/0.7 over quarter cells 0..2, and the bilinear upsample blends it
    with 0.6 over the last quarter column/row."""
    a, d, p = _frames()
    b = a.copy()
    b[0, 6, 5, 0] = 255 - a[0, 6, 5, 0] if a[0, 6, 5, 0] < 128 else 0
    delta = abs(int(b[0, 6, 5, 0]) - int(a[0, 6, 5, 0])) / 255.0
    hi = BETA + (delta / 16.0) / LAM
    out, m = oracle_mod.refine_depth_soft(b, a, d, p)
    assert m[0, 0, 0] == pytest.approx(hi, rel=1e-14)
    assert m[0, 9, 9] == pytest.approx(hi, rel=1e-14)
    # x = 10: sample 2.125 between quarter columns 2 (hi) and 3 (beta)
    assert m[0, 5, 10] == pytest.approx(0.875 * hi + 0.125 * BETA, rel=1e-14)
    assert m[0, 15, 15] == pytest.approx(BETA, rel=1e-14)
    i = (5, 10)
    np.testing.assert_allclose(out[0][i], m[0][i] * d[0][i] + (1 - m[0][i]) * p[0][i], rtol=1e-14)


def test_invalid_depths(oracle_mod):
    a, d, p = _frames()
    d[0, 1, 1] = 0.0
    p[0, 2, 2] = np.nan
    out, m = oracle_mod.refine_depth_soft(a, a, d, p)
    assert out[0, 1, 1] == p[0, 1, 1]
    assert out[0, 2, 2] == d[0, 2, 2]


def test_odd_sizes_average_partial_blocks(oracle_mod):
    a, d, p = _frames(H=9, W=13)
    b = a.copy()
    b[0, 8, 12, 2] = 255 if a[0, 8, 12, 2] < 128 else 0     # alone in its partial 1x1 quarter cell
    delta = abs(int(b[0, 8, 12, 2]) - int(a[0, 8, 12, 2])) / 255.0
    out, m = oracle_mod.refine_depth_soft(b, a, d, p)
    assert m[0, 8, 12] == pytest.approx(min(BETA + delta / LAM, 1.0), rel=1e-14)
