"""Pins of the oracle's uniform-blend loss (Sec. 3.3's 0.8 L1 + 0.1 L_Depth on the blend
of Eq. 4 with unit weights): a two-view, three-pixel case worked by hand, the single-view
reduction, and its gradients against central finite differences of the loss itself on
seeded inputs away from the kinks of |x|."""
import numpy as np


def test_worked_by_hand(oracle_mod):
    # two views, 1 x 3 pixels; channel values chosen so every term is exact in binary
    I = np.zeros((2, 1, 3, 3))
    I[0, 0, 0] = [0.5, 0.25, 1.0]
    I[1, 0, 0] = [0.25, 0.25, 0.0]     # pixel 0: both views, B = [0.375, 0.25, 0.5]
    I[0, 0, 1] = [1.0, 0.0, 0.5]       # pixel 1: view 0 only, B = [1, 0, 0.5]
    a = np.array([[[1, 1, 0]], [[1, 0, 0]]], np.float64)   # pixel 2: no view
    D = np.array([[[2.0, 3.0, 9.0]], [[4.0, 7.0, 9.0]]])
    F = np.array([[2.5, 3.5, 1.0]])
    gt = np.array([[[0.5, 0.5, 0.5], [0.75, 0.25, 0.25], [0.0, 0.0, 0.0]]])
    L, L1, LD, g = oracle_mod.uniform_blend_loss(I, a, D, F, gt)
    # |B - GT|: pixel 0 -> 0.125 + 0.25 + 0 ; pixel 1 -> 0.25 + 0.25 + 0.25 ; n = 2 covered
    assert L1 == (0.375 + 0.75) / 6.0
    # Dbar: pixel 0 -> 3, pixel 1 -> 3 ; |F - Dbar| = 0.5 + 0.5 ; K H W = 6
    assert LD == 1.0 / 6.0
    assert L == 0.8 * L1 + 0.1 * LD
    assert np.array_equal(g["rgb"][0, 0], 0.8 / 6.0 * np.array([-1.0, -1.0, 0.0]) * 0.5)
    assert np.array_equal(g["rgb"][0, 1], 0.8 / 6.0 * np.array([1.0, -1.0, 1.0]))
    assert np.array_equal(g["rgb"][0, 2], np.zeros(3))
    # F - Dbar = -0.5 at pixel 0 (d|.|/dDbar = +1, split over its 2 views), +0.5 at pixel 1
    assert np.allclose(g["depth"][0], [0.1 / 6.0 * 0.5, -0.1 / 6.0, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(g["fused"][0], [-0.1 / 6.0, 0.1 / 6.0, 0.0], rtol=0, atol=1e-15)


def test_single_view_is_the_plain_l1(oracle_mod):
    rng = np.random.default_rng(3)
    I = rng.random((1, 5, 7, 3))
    a = np.ones((1, 5, 7))
    gt = rng.random((5, 7, 3))
    D = rng.random((1, 5, 7)) + 1
    L, L1, LD, _ = oracle_mod.uniform_blend_loss(I, a, D, D[0], gt)
    assert abs(L1 - np.abs(I[0] - gt).mean()) < 1e-15
    assert LD == 0.0


def test_gradients_match_central_differences(oracle_mod):
    rng = np.random.default_rng(11)
    K, H, W = 3, 6, 5
    I = rng.random((K, H, W, 3))
    a = (rng.random((K, H, W)) < 0.7).astype(np.float64)
    D = rng.random((K, H, W)) * 2 + 1
    F = rng.random((H, W)) * 2 + 1
    F[0, 0] = 0.0                       # no fused depth: no L_Depth term there
    gt = rng.random((H, W, 3))
    L0, _, _, g = oracle_mod.uniform_blend_loss(I, a, D, F, gt)
    h = 1e-7
    checked = 0
    for k, y, x, c in [(k, y, x, c) for k in range(K) for y in range(H) for x in range(W) for c in range(3)]:
        Ip, Im = I.copy(), I.copy()
        Ip[k, y, x, c] += h
        Im[k, y, x, c] -= h
        fd = (oracle_mod.uniform_blend_loss(Ip, a, D, F, gt)[0] - oracle_mod.uniform_blend_loss(Im, a, D, F, gt)[0]) / (2 * h)
        assert abs(fd - a[k, y, x] * g["rgb"][y, x, c]) < 1e-7, (k, y, x, c)
        checked += 1
    for k in range(K):
        for y in range(H):
            for x in range(W):
                Dp, Dm = D.copy(), D.copy()
                Dp[k, y, x] += h
                Dm[k, y, x] -= h
                fd = (oracle_mod.uniform_blend_loss(I, a, Dp, F, gt)[0] - oracle_mod.uniform_blend_loss(I, a, Dm, F, gt)[0]) / (2 * h)
                assert abs(fd - a[k, y, x] * g["depth"][y, x]) < 1e-7, (k, y, x)
    for y in range(H):
        for x in range(W):
            if F[y, x] <= 0:
                continue
            Fp, Fm = F.copy(), F.copy()
            Fp[y, x] += h
            Fm[y, x] -= h
            fd = (oracle_mod.uniform_blend_loss(I, a, D, Fp, gt)[0] - oracle_mod.uniform_blend_loss(I, a, D, Fm, gt)[0]) / (2 * h)
            assert abs(fd - g["fused"][y, x]) < 1e-7, (y, x)
    assert checked == K * H * W * 3
