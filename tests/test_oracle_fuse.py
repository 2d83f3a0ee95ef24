"""Pins for the oracle's confidence weight and TSDF fusion (Supplement A.1, Eq. 3).

Each expected value below is derived by hand for a constructed configuration
(flat or stepped depth, identity camera, fronto-parallel planes, an occluding
wall) or comes from the analytic ray caster, so that a dropped term, a wrong
sign, a transposed operand or a wrong index fails one of them.
"""
import math

import numpy as np
import pytest

MU = 0.04


def test_weight_flat_is_one(oracle_mod):
    d = np.full((20, 30), 2.0, np.float32)
    for (u, v) in [(0, 0), (15, 10), (29, 19), (3, 17)]:
        assert oracle_mod.weight(d, u, v, MU) == 1.0


def test_weight_checkerboard_step(oracle_mod):
    # step of 0.1 >= mu: every unlike neighbour contributes mu^2; an interior
    # 7x7 window holds 24 unlike cells -> nu = 24 mu^2 -> omega = 0.001*7/(mu*sqrt(24))
    u, v = np.meshgrid(np.arange(30), np.arange(20))
    d = (2.0 + 0.1 * ((u + v) % 2)).astype(np.float32)
    w = oracle_mod.weight(d, 12, 9, MU)
    assert w == pytest.approx(0.007 / (MU * math.sqrt(24)), rel=1e-12)


def test_weight_border_replicates(oracle_mod):
    # only pixel (0,0) differs; at (0,0) the clamped window maps 16 cells onto
    # (0,0) itself and 33 onto unlike pixels; at (1,1) it maps 9 cells onto (0,0)
    d = np.full((20, 30), 2.0, np.float32)
    d[0, 0] = 2.5
    assert oracle_mod.weight(d, 0, 0, MU) == pytest.approx(0.007 / (MU * math.sqrt(33)), rel=1e-12)
    assert oracle_mod.weight(d, 1, 1, MU) == pytest.approx(0.007 / (MU * 3.0), rel=1e-12)


def test_weight_small_variation_and_invalid(oracle_mod):
    d = np.full((20, 30), 2.0, np.float32)
    d[5, 5] = np.float32(2.01)          # below mu: contributes its square
    nu = (float(np.float32(2.01)) - 2.0) ** 2
    assert oracle_mod.weight(d, 6, 6, MU) == pytest.approx(min(0.001 * (nu / 49) ** -0.5, 1.0), rel=1e-12)
    d[5, 5] = np.nan                    # invalid neighbour: maximal variation mu^2
    assert oracle_mod.weight(d, 6, 6, MU) == pytest.approx(0.007 / MU, rel=1e-12)
    assert oracle_mod.weight(d, 5, 5, MU) == 0.0   # invalid centre
    d[5, 5] = 0.0
    assert oracle_mod.weight(d, 5, 5, MU) == 0.0


def _smooth_depth(H, W, seed, lo=1.5, hi=3.5):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W] / max(H, W)
    f = np.zeros((H, W))
    for _ in range(4):
        a, b, c = rng.uniform(-6, 6, 3)
        f += np.sin(a * x + b * y + c)
    f = (f - f.min()) / (f.max() - f.min())
    return (lo + (hi - lo) * f).astype(np.float32)


@pytest.mark.parametrize("deg", [0.0, 13.0])
def test_identity_camera_reproduces_depth(oracle_mod, synth_mod, deg):
    """Target = input camera, one view, samples finer than mu: each bracketing
    sample is inside the band, so the interpolated crossing is the input depth."""
    from synth.configs import arc_cameras
    cam = arc_cameras(64, 48, [deg])[0]
    d = _smooth_depth(48, 64, seed=3)
    r = oracle_mod.fuse_depth([cam], d[None], cam, 160, 0.5, 5.0, 0.05)
    assert (r["index"] >= 0).all()
    np.testing.assert_allclose(r["depth"], d.astype(np.float64), rtol=1e-9, atol=0)


def _translation_rig(W, H, offsets):
    from synth import camera_at
    return [camera_at(W, H, (ox, oy, 0.0)) for ox, oy in offsets]


def test_fronto_parallel_plane_fine_sampling(oracle_mod, synth_mod):
    """Every view sees depth d everywhere; with sample spacing below mu the fused depth is d."""
    from synth import camera_at
    offs = [(-0.1, 0.0), (0.1, 0.0), (0.0, -0.05), (0.0, 0.05)]
    cams = _translation_rig(96, 64, offs)
    tgt = camera_at(96, 64, (0.0, 0.0, 0.0))
    for d in [1.1, 2.0, 2.9371]:
        dep = np.full((4, 64, 96), d, np.float32)
        r = oracle_mod.fuse_depth(cams, dep, tgt, 257, 0.5, 5.0, MU)
        inner = (slice(12, -12), slice(12, -12))
        assert (r["index"][inner] >= 0).all()
        np.testing.assert_allclose(r["depth"][inner], float(np.float32(d)), rtol=1e-9)


def test_fronto_parallel_plane_coarse_sampling(oracle_mod, synth_mod):
    """Sample spacing above mu: by hand, with c(z) = (d - z)/mu and every view
    cut off beyond z = d + mu, the crossing exists iff some sample lies in
    [d, d + mu], and then D = z_s + dz * c_s / (c_s - c_{s+1})."""
    from synth import camera_at
    cams = _translation_rig(64, 48, [(-0.05, 0.0), (0.05, 0.0)])
    tgt = camera_at(64, 48, (0.0, 0.0, 0.0))
    D, zn, zf = 64, 0.5, 5.0
    dz32 = np.float32((np.float32(zf) - np.float32(zn)) / np.float64(D - 1))
    # sample positions z_s = fma(s, dz, zn) in FP32: the product and sum are exact in FP64, one rounding
    zs = np.array([np.float32(float(np.float32(s)) * float(dz32) + float(np.float32(zn))) for s in range(D)],
                  np.float64)
    holes = 0
    for d in np.linspace(1.2, 3.2, 23):
        d32 = float(np.float32(d))
        dep = np.full((2, 48, 64), d32, np.float32)
        r = oracle_mod.fuse_depth(cams, dep, tgt, D, zn, zf, MU)
        c = (d32 - zs) / float(np.float32(MU))
        expect_s = -1
        for s in range(D - 1):
            if c[s] > 0 and c[s + 1] <= 0 and c[s + 1] >= -1:
                expect_s = s
                break
        px = r["index"][24, 32]
        assert px == expect_s
        if expect_s < 0:
            holes += 1
            assert r["depth"][24, 32] == 0.0
        else:
            cs, cs1 = min(c[expect_s], 1.0), c[expect_s + 1]
            exp = zs[expect_s] + (zs[expect_s + 1] - zs[expect_s]) * cs / (cs - cs1)
            assert r["depth"][24, 32] == pytest.approx(exp, rel=1e-9)
    assert 0 < holes < 23   # spacing 0.071 > mu: some depths fall between samples


def test_occluding_wall_is_cut_off(oracle_mod, synth_mod):
    """View 0 sees a wall at 1.0, view 1 sees a wall at 3.0.  Behind z = 1 + mu
    view 0 drops out (omega = 0 where sdf < -1), so the only crossing is view 1's
    surface at 3.0; were the occluded view kept at -1, S would reach 0 near 1.04."""
    from synth import camera_at
    cams = _translation_rig(64, 48, [(-0.02, 0.0), (0.02, 0.0)])
    tgt = camera_at(64, 48, (0.0, 0.0, 0.0))
    dep = np.stack([np.full((48, 64), 1.0, np.float32), np.full((48, 64), 3.0, np.float32)])
    r = oracle_mod.fuse_depth(cams, dep, tgt, 450, 0.5, 5.0, MU)
    inner = (slice(8, -8), slice(8, -8))
    np.testing.assert_allclose(r["depth"][inner], 3.0, rtol=1e-9)


def test_no_surface_cases(oracle_mod, synth_mod):
    from synth import camera_at
    cams = _translation_rig(32, 24, [(-0.05, 0.0), (0.05, 0.0)])
    tgt = camera_at(32, 24, (0.0, 0.0, 0.0))
    for fill in [0.2, 9.0, 0.0, np.nan, np.inf]:    # before near, beyond far, invalid
        dep = np.full((2, 24, 32), fill, np.float32)
        r = oracle_mod.fuse_depth(cams, dep, tgt, 32, 0.5, 5.0, MU)
        assert (r["index"] == -1).all() and (r["depth"] == 0.0).all()


def test_view_permutation_invariance(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(64, 48, 4, 48)
    _, d = w.render_inputs(0)
    a = oracle_mod.fuse_depth(w.inputs, d, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu)
    perm = [2, 0, 3, 1]
    b = oracle_mod.fuse_depth([w.inputs[k] for k in perm], d[perm], w.targets[0], w.num_samples,
                              w.z_near, w.z_far, w.mu)
    ok = (a["ambiguous"] == 0) & (b["ambiguous"] == 0)
    assert np.array_equal(a["index"][ok], b["index"][ok])
    np.testing.assert_allclose(a["depth"][ok], b["depth"][ok], rtol=1e-12)


def test_normalize_keeps_crossing_index(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(64, 48, 3, 40)
    _, d = w.render_inputs(0)
    a = oracle_mod.fuse_depth(w.inputs, d, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu)
    b = oracle_mod.fuse_depth(w.inputs, d, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu, normalize=True)
    ok = (a["ambiguous"] == 0) & (b["ambiguous"] == 0)
    assert np.array_equal(a["index"][ok], b["index"][ok])


@pytest.mark.parametrize("rig", ["arc", "translation"])
def test_converges_to_ray_cast_depth(oracle_mod, synth_mod, rig):
    """Fine sampling on a noise-free scene: the fused depth approaches the
    analytic first hit along the target ray, up to the nearest-pixel error."""
    from synth import camera_at, configs, render
    if rig == "arc":
        w = configs.plain_320x240()
        from synth.configs import arc_cameras
        ins = arc_cameras(160, 120, [-15, -5, 5, 15])
        tgt = arc_cameras(160, 120, [2.0])[0]
        zn, zf = 0.5, 5.0
    else:
        w = configs.video_8x720p()
        from synth.configs import rig_2x4
        ins = rig_2x4(160, 90)
        tgt = camera_at(160, 90, (0.03, 0.02, 0.0))
        zn, zf = 0.3, 8.0
    sc = w.scene(0)
    d = np.stack([render(sc, c)[1] for c in ins])
    _, gt = render(sc, tgt)
    D = int((zf - zn) / 0.005) + 1
    r = oracle_mod.fuse_depth(ins, d, tgt, D, zn, zf, 0.02)
    # away from depth edges of the ground truth
    gy, gx = np.gradient(gt.astype(np.float64))
    smooth = (np.abs(gx) + np.abs(gy) < 0.02 * gt) & (gt > zn) & (gt < zf)
    found = (r["index"] >= 0) & smooth
    assert found.sum() > 0.8 * smooth.sum()
    err = np.abs(r["depth"][found] - gt[found]) / gt[found]
    assert np.median(err) < 2e-3
    assert np.percentile(err, 95) < 1e-2
