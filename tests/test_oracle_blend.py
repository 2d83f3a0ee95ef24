"""Pins for the oracle's network input (the supplement's list of the (9K + 1)
channels) and the blend of Eqs. 4-5 with L_Depth.

Closed forms: a fronto-parallel plane (normal towards the camera, the ray
dot products of a view displaced sideways), a tilted plane (the normal of the
finite differences equals the plane's), camera distances and axis dot
products, channel copies, invalid neighbours; the blend by hand for one and
two views, the background weight's two ends and L_Depth on a 2-pixel case.
"""
import math

import numpy as np
import pytest


def _cam(W, H, centre=(0.0, 0.0, 0.0), R=None):
    from synth import Camera
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    return Camera(W, H, 100.0, 100.0, 15.0, 10.0, R, -R @ np.asarray(centre, np.float64))


def _inputs(K, H, W, seed=0):
    rng = np.random.default_rng(seed)
    rgba = rng.integers(0, 2 ** 32, size=(K, H, W), dtype=np.uint64).astype(np.uint32)
    depth = rng.uniform(1.0, 3.0, size=(K, H, W)).astype(np.float32)
    alpha = (rng.random((K, H, W)) > 0.2).astype(np.uint8)
    return rgba, depth, alpha


def test_channel_copies_and_camera_maps(oracle_mod, synth_mod):
    tgt = _cam(31, 21)
    views = [_cam(31, 21, (0.3, 0.0, 0.0)), _cam(31, 21, (0.0, -0.4, 0.1))]
    rgba, depth, alpha = _inputs(2, 21, 31)
    fused = np.full((21, 31), 2.0, np.float32)
    f = oracle_mod.blend_features(views, tgt, rgba, depth, alpha, fused)
    K = 2
    assert f.shape == (9 * K + 1, 21, 31)
    for k in range(K):
        for ch in range(3):
            assert np.array_equal(f[3 * k + ch], ((rgba[k] >> (8 * ch)) & 0xff) / 255.0)
        assert np.array_equal(f[3 * K + k], depth[k].astype(np.float64))
        assert np.array_equal(f[4 * K + k], alpha[k].astype(np.float64))
    assert np.array_equal(f[5 * K], fused.astype(np.float64))
    np.testing.assert_allclose(f[7 * K + 1], 0.3, atol=1e-12)
    np.testing.assert_allclose(f[7 * K + 2], math.sqrt(0.4 ** 2 + 0.1 ** 2), atol=1e-12)
    np.testing.assert_allclose(f[8 * K + 1:8 * K + 3], 1.0, atol=1e-12)   # parallel optical axes


def test_fronto_parallel_plane(oracle_mod, synth_mod):
    """Plane at depth 2 facing the target: n = (0, 0, -1).  At the principal point
    (15, 10) P = (0, 0, 2); a view at (b, 0, 0) gives d = (-b, 0, 2) / sqrt(b^2 + 4), so
    n . d = -2 / sqrt(b^2 + 4) and r_t . d = 2 / sqrt(b^2 + 4)."""
    b = 0.5
    tgt = _cam(31, 21)
    views = [_cam(31, 21, (b, 0.0, 0.0))]
    rgba, depth, alpha = _inputs(1, 21, 31)
    fused = np.full((21, 31), 2.0, np.float32)
    f = oracle_mod.blend_features(views, tgt, rgba, depth, alpha, fused)
    nd, rd = f[6, 10, 15], f[7, 10, 15]
    assert nd == pytest.approx(-2.0 / math.sqrt(b * b + 4.0), abs=1e-12)
    assert rd == pytest.approx(2.0 / math.sqrt(b * b + 4.0), abs=1e-12)
    # the image border has no central differences: normal feature 0 there, ray feature still set
    assert f[6, 0, 15] == 0.0 and f[6, 10, 30] == 0.0 and f[7, 0, 15] != 0.0


def test_tilted_plane_normal(oracle_mod, synth_mod):
    """Plane n_w . X = 2 with n_w = (0.3, -0.2, 1)/|.| in the target frame: D(i, j) =
    2 / (n_w . K^-1 [i, j, 1]).  With a view at the target's own centre, n . d_k = n . r_t
    = -|n_w . r_t| (the normal turned towards the camera)."""
    tgt = _cam(31, 21)
    nw = np.array([0.3, -0.2, 1.0])
    nw /= np.linalg.norm(nw)
    jj, ii = np.mgrid[0:21, 0:31].astype(np.float64)
    ray = np.stack([(ii - 15.0) / 100.0, (jj - 10.0) / 100.0, np.ones_like(ii)], -1)
    D = 2.0 / (ray @ nw)
    rgba, depth, alpha = _inputs(1, 21, 31)
    f = oracle_mod.blend_features([tgt], tgt, rgba, depth, alpha, D.astype(np.float32))
    r = ray / np.linalg.norm(ray, axis=-1, keepdims=True)
    expect = -np.abs(r @ nw)
    np.testing.assert_allclose(f[6, 1:-1, 1:-1], expect[1:-1, 1:-1], atol=2e-4)
    np.testing.assert_allclose(f[7, 1:-1, 1:-1], 1.0, atol=1e-12)   # view ray = target ray


def test_invalid_depth_zeroes_geometry(oracle_mod, synth_mod):
    tgt = _cam(31, 21)
    views = [_cam(31, 21, (0.2, 0.0, 0.0))]
    rgba, depth, alpha = _inputs(1, 21, 31)
    fused = np.full((21, 31), 2.0, np.float32)
    fused[10, 15] = 0.0
    f = oracle_mod.blend_features(views, tgt, rgba, depth, alpha, fused)
    assert f[6, 10, 15] == 0.0 and f[7, 10, 15] == 0.0     # no point at p
    assert f[6, 10, 14] == 0.0 and f[6, 9, 15] == 0.0      # a neighbour without depth
    assert f[7, 10, 14] != 0.0 and f[6, 10, 13] != 0.0


def test_blend_by_hand(oracle_mod, synth_mod):
    """Two views, two pixels.  Pixel 0: colours 200 and 100 (red), weights 0.75 and 0.25,
    both alpha 1 -> I_FG = (0.75 * 200 + 0.25 * 100) / 255; w_BG = 0.2 mixes 0.2 of I_BG.
    Pixel 1: view 0 alpha 0 -> only view 1; w_BG = 1 -> I = I_BG exactly.
    L_Depth = (|3 - (0.75 * 2 + 0.25 * 4)| + |5 - 4|) / (2 * 2) = (0.5 + 1) / 4."""
    rgba = np.array([[[200, 50]], [[100, 100]]], np.uint32)
    alpha = np.array([[[1, 0]], [[1, 1]]], np.uint8)
    wd = np.array([[[2.0, 9.0]], [[4.0, 4.0]]], np.float32)
    fused = np.array([[3.0, 5.0]], np.float32)
    w = np.array([[[0.75, 0.6]], [[0.25, 0.3]]])
    w_bg = np.array([[0.2, 1.0]])
    i_bg = np.stack([np.full((1, 2), 0.5), np.full((1, 2), 0.1), np.full((1, 2), 0.9)])
    img, L = oracle_mod.blend(rgba, alpha, wd, fused, w, w_bg, i_bg)
    fg0 = (0.75 * 200 + 0.25 * 100) / 255.0
    assert img[0, 0, 0] == pytest.approx(0.8 * fg0 + 0.2 * 0.5, abs=1e-15)
    assert img[1, 0, 0] == pytest.approx(0.2 * 0.1, abs=1e-15)        # green channel is 0 in both views
    assert img[:, 0, 1] == pytest.approx([0.5, 0.1, 0.9], abs=1e-15)
    assert L == pytest.approx((0.5 + 1.0) / 4.0, abs=1e-15)
    # no view at a pixel: the foreground is 0
    img, _ = oracle_mod.blend(rgba, np.zeros_like(alpha), wd, fused, w, np.zeros((1, 2)), i_bg)
    assert np.all(img == 0.0)
