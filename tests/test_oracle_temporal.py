"""Pins for the temporal term (Sec. 3.2, Supplement A.2) in the oracle.

* the weight, worked by hand for constructed winners and masks;
* with zero temporal weight the fusion is the plain fusion;
* a plane seen by K views at d1 with the previous output at d2 (within the
  band, fine sampling): S is linear in z, so the fused depth is the weighted
  mean (K d1 + w d2) / (K + w) exactly, and the views' weight at the crossing
  is K (flat depth: every confidence weight is 1).
"""
import numpy as np
import pytest


def test_temporal_weight_by_hand(oracle_mod):
    # 2 views of 2x2 pixels, target 3x1
    masks = np.array([[[0.2, 0.9], [0.5, 1.0]], [[0.7, 0.6], [0.1, 0.3]]], np.float32)
    winner = np.array([[[0, 3, -1]], [[1, -1, -1]]], np.int32)
    wp = np.array([[2.0, 1.0, 5.0]], np.float32)
    wv = np.array([[3.0, 2.0, 4.0]], np.float32)
    w, M = oracle_mod.temporal_weight(masks, winner, wp, wv, beta_t=1.5, eta=15.0)
    # pixel 0: max(0.2 (view 0, pixel 0), 0.6 (view 1, pixel 1)) = 0.6
    # pixel 1: view 0 pixel 3 -> 1.0;  pixel 2: no winner -> 1
    np.testing.assert_allclose(M[0], [0.6, 1.0, 1.0], rtol=1e-7)
    np.testing.assert_allclose(w[0], [min(1.5 * 5.0 * (1 - float(np.float32(0.6))), 15.0), 0.0, 0.0], rtol=1e-7)
    w2, _ = oracle_mod.temporal_weight(np.zeros_like(masks), winner[:, :, :1], wp[:, :1] * 10, wv[:, :1], 1.0, 15.0)
    assert w2[0, 0] == 15.0   # capped at eta


def test_zero_weight_is_plain_fusion(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(40, 30, 3, 96)
    _, d = w.render_inputs(0)
    t = w.targets[0]
    plain = oracle_mod.fuse_depth(w.inputs, d, t, w.num_samples, w.z_near, w.z_far, w.mu)
    tz = oracle_mod.fuse_depth_temporal(w.inputs, d, t, w.num_samples, w.z_near, w.z_far, w.mu,
                                        np.full((30, 40), 2.0, np.float32), np.zeros((30, 40), np.float32))
    assert np.array_equal(plain["index"], tz["index"])
    assert np.array_equal(plain["depth"], tz["depth"])


def test_plane_weighted_mean(oracle_mod, synth_mod):
    from synth import camera_at
    cams = [camera_at(48, 32, (x, y, 0.0)) for x, y in [(-0.05, 0.0), (0.05, 0.0), (0.0, 0.04)]]
    tgt = camera_at(48, 32, (0.0, 0.0, 0.0))
    d1, d2, wt = 2.5, 2.52, 4.0
    dep = np.full((3, 32, 48), d1, np.float32)
    r = oracle_mod.fuse_depth_temporal(cams, dep, tgt, 1024, 0.5, 5.0, 0.05, np.full((32, 48), d2, np.float32),
                                       np.full((32, 48), wt, np.float32))
    inner = (slice(6, -6), slice(8, -8))
    exp = (3 * float(np.float32(d1)) + wt * float(np.float32(d2))) / (3 + wt)
    np.testing.assert_allclose(r["depth"][inner], exp, rtol=1e-9)
    np.testing.assert_allclose(r["wview"][inner], 3.0, rtol=1e-12)
