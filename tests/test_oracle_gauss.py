"""Pins for the oracle's pixel-sized Gaussian render (Sec. 3.1, Supplement A.3;
rasterisation rules of 3D Gaussian splatting).

Hand-worked values for one Gaussian (on and off the optical axis, which pins
the EWA covariance including the sign of its off-diagonal term), the radius
cap, front-to-back order and early termination on a stack of six Gaussians,
and a uniform-colour plane (colour = c x opacity, depth = the plane's).
"""
import math

import numpy as np
import pytest


def _cam(W=32, H=24, x=0.0):
    from synth import Camera
    return Camera(W, H, 100.0, 100.0, 10.0, 8.0, np.eye(3), np.array([-x, 0.0, 0.0]))


def _one(oracle_mod, u, v, d=2.0, scale_px=0.5, max_radius=8, colour=0x00c08040):
    cam = _cam()
    dep = np.zeros((1, cam.height, cam.width), np.float32)
    dep[0, v, u] = d
    rgb = np.full((1, cam.height, cam.width), colour, np.uint32)
    return oracle_mod.gauss_splat([cam], dep, rgb, cam, scale_px=scale_px, max_radius=max_radius)


def test_single_gaussian_on_axis(oracle_mod, synth_mod):
    """Source = target camera, one valid pixel at the principal point (10, 8):
    rho = 1, a = b = 0, Sigma = (0.25 + 0.3) I = 0.55 I; radius ceil(3 sqrt(0.55 + sqrt(0.1))) = 3.
    alpha at offset (dx, dy) = min(0.99, exp(-(dx^2 + dy^2) / 1.1))."""
    r = _one(oracle_mod, 10, 8)
    a = r["color"][0, ..., 3]
    red = r["color"][0, ..., 0]
    expect = {(10, 8): 0.99,                     # clamped
              (11, 8): 0.4028903215, (9, 8): 0.4028903215, (10, 9): 0.4028903215,
              (11, 9): 0.1623206112,              # exp(-2 / 1.1)
              (12, 8): 0.0263479808,              # exp(-4 / 1.1) >= 1/255
              (13, 8): 0.0,                       # exp(-9 / 1.1) = 2.8e-4 < 1/255: skipped
              (14, 8): 0.0}                       # outside the radius
    for (i, j), e in expect.items():
        assert a[j, i] == pytest.approx(e, abs=2e-7), (i, j)
        assert red[j, i] == pytest.approx(e * 0x40 / 255.0, abs=2e-7)
    assert r["depth"][0, 8, 10] == pytest.approx(2.0, rel=1e-7)
    assert r["depth"][0, 8, 13] == 0.0
    # every pixel with alpha >= 1/255 inside the radius: squared offsets 0, 1, 2, 4, 5 (8 of those);
    # offsets 8 and 9 fall below 1/255
    assert a.sum() == pytest.approx(0.99 + 4 * 0.4028903215 + 4 * 0.1623206112 + 4 * 0.0263479808
                                    + 8 * math.exp(-5 / 1.1), abs=1e-6)


def test_radius_cap(oracle_mod, synth_mod):
    """max_radius = 1 drops the offset-2 pixel although its alpha is above 1/255."""
    r = _one(oracle_mod, 10, 8, max_radius=1)
    a = r["color"][0, ..., 3]
    assert a[8, 11] == pytest.approx(0.4028903215, abs=2e-7)
    assert a[8, 12] == 0.0 and a[9, 11] == pytest.approx(0.1623206097, abs=2e-7)


def test_single_gaussian_off_axis(oracle_mod, synth_mod):
    """Pixel (60, 48): a = 0.5, b = 0.4; Sigma = 0.25 [[1.25, 0.2], [0.2, 1.16]] + 0.3 I
    = [[0.6125, 0.05], [0.05, 0.59]], det 0.358875, conic (0.59, -0.05, 0.6125) / det.
    power = -0.5 (cxx dx^2 + cyy dy^2) - cxy dx dy gives alpha(dx=-1, dy=-1) = exp(-1.5361)
    and alpha(dx=-1, dy=+1) = exp(-1.8147)."""
    cam = _cam(96, 64)
    dep = np.zeros((1, 64, 96), np.float32)
    dep[0, 48, 60] = 3.0
    rgb = np.full((1, 64, 96), 0xffffffff, np.uint32)
    r = oracle_mod.gauss_splat([cam], dep, rgb, cam)
    a = r["color"][0, ..., 3]
    det = 0.6125 * 0.59 - 0.05 ** 2
    cxx, cxy, cyy = 0.59 / det, -0.05 / det, 0.6125 / det
    assert a[49, 61] == pytest.approx(0.2152295477, abs=1e-6)   # pixel (61, 49): dx = dy = -1
    assert a[47, 61] == pytest.approx(0.1628869770, abs=1e-6)   # pixel (61, 47): dx = -1, dy = +1
    assert a[49, 61] == pytest.approx(math.exp(-0.5 * (cxx + cyy) - cxy), abs=1e-6)
    assert a[47, 61] == pytest.approx(a[49, 59], abs=1e-9) and a[49, 61] == pytest.approx(a[47, 59], abs=1e-9)


def test_front_to_back_order_and_termination(oracle_mod, synth_mod):
    """Source shifted by 0.12 m along x (fx = 100): u_t = u_s + 12 / d.  Six source
    pixels u_s = 0..5 on row 8 with d = 12 / (12.5 - u_s) all land on x = 12.5, so target
    pixel (12, 8) sees six Gaussians at dx = 0.5, nearest first in u_s order.  Each has
    alpha = exp(-0.125 / Sxx), Sxx = 0.25 (1 + 0.025^2) + 0.3; the sixth would take T
    below 1e-4 and stops the walk."""
    src, tgt = _cam(x=0.12), _cam()
    dep = np.zeros((1, 24, 32), np.float32)
    rgb = np.zeros((1, 24, 32), np.uint32)
    for u in range(6):
        dep[0, 8, u] = 12.0 / (12.5 - u)
        rgb[0, 8, u] = 40 * (u + 1)             # red channel
    r = oracle_mod.gauss_splat([src], dep, rgb, tgt)
    al = math.exp(-0.125 / (0.25 * (1 + 0.025 ** 2) + 0.3))
    T = [(1 - al) ** n for n in range(7)]
    assert T[5] >= 1e-4 > T[6]
    red = sum(40 * (u + 1) / 255.0 * al * T[u] for u in range(5))
    depth = sum(dep[0, 8, u] * al * T[u] for u in range(5)) / sum(al * T[u] for u in range(5))
    c = r["color"][0, 8, 12]
    assert c[0] == pytest.approx(red, rel=1e-5)
    assert c[3] == pytest.approx(1 - T[5], rel=1e-6)
    assert r["depth"][0, 8, 12] == pytest.approx(depth, rel=1e-5)
    # the other side of the stack (dx = -0.5) is identical
    assert r["color"][0, 8, 13] == pytest.approx(c, rel=1e-6)
    assert r["ambiguous"][0, 8, 12] == 0


def test_uniform_plane(oracle_mod, synth_mod):
    """A fronto-parallel plane at depth 2 in one constant colour seen with parallax:
    colour = c x opacity and depth = 2 wherever anything lands."""
    src, tgt = _cam(48, 32, x=0.05), _cam(48, 32)
    dep = np.full((1, 32, 48), 2.0, np.float32)
    rgb = np.full((1, 32, 48), 0x00336699, np.uint32)
    r = oracle_mod.gauss_splat([src], dep, rgb, tgt)
    col, a = r["color"][0], r["color"][0, ..., 3]
    for ch, v in enumerate((0x99, 0x66, 0x33)):
        np.testing.assert_allclose(col[..., ch], v / 255.0 * a, atol=1e-12)
    m = a > 0
    assert m.mean() > 0.8 and a[m].max() <= 1.0 - 1e-4
    np.testing.assert_allclose(r["depth"][0][m], 2.0, rtol=1e-12)


def test_pixel_subset_matches_full(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(40, 30, 2, 16)
    rgb, d = w.render_inputs(0)
    u = np.ascontiguousarray(rgb).view(np.uint32)[..., 0]
    full = oracle_mod.gauss_splat(w.inputs, d, u, w.targets[0])
    px = np.array([0, 17, 333, 40 * 30 - 1, 600], np.int32)
    sub = oracle_mod.gauss_splat(w.inputs, d, u, w.targets[0], pixels=px)
    assert np.array_equal(sub["color"], full["color"].reshape(2, -1, 4)[:, px])
    assert np.array_equal(sub["depth"], full["depth"].reshape(2, -1)[:, px])
