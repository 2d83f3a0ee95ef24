"""Degenerate and extreme shapes through every entry point, against the oracle:
1x1 and single-row / single-column targets (crops of a real target camera),
two samples per ray, the maximum of 32 views, and a 1x1 input."""
import numpy as np
import pytest
import torch

from gpu_util import compare_fused, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvs():
    assert torch.cuda.is_available()
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


def _crop(cam, i0, j0, w, h):
    """The w x h window of `cam` starting at pixel (i0, j0), as a camera of its own."""
    from synth import Camera
    return Camera(w, h, cam.fx, cam.fy, cam.cx - i0, cam.cy - j0, cam.R, cam.t)


CROPS = [(35, 22, 1, 1), (0, 10, 70, 1), (12, 0, 1, 45), (60, 40, 10, 5)]


@pytest.mark.parametrize("crop", CROPS)
def test_fuse_and_splat_on_crops(gvs, oracle_mod, crop):
    from synth import configs
    w = configs.tiny(70, 45, 3, 96)
    rgb, d = w.render_inputs(0)
    tgt = _crop(w.targets[0], *crop)
    fused, cross = gvs.fuse_depth(w.inputs, to_dev(d), tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(w.inputs, to_dev(d), to_dev(u32(rgb)), tgt, fused=fused, mu_guide=w.mu)
    torch.cuda.synchronize()
    ref = oracle_mod.fuse_depth(w.inputs, d, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    compare_fused(fused, cross, ref)
    rs = oracle_mod.forward_splat(w.inputs, d, u32(rgb), tgt, mu_guide=w.mu,
                                  fused=fused.cpu().numpy().astype(np.float64))
    assert np.array_equal(sp["winner"].cpu().numpy(), rs["winner"])
    assert np.array_equal(sp["guided"].cpu().numpy(), rs["guided"])


@pytest.mark.parametrize("crop", CROPS)
def test_gauss_sphere_features_on_crops(gvs, oracle_mod, crop):
    from synth import configs
    w = configs.tiny(70, 45, 3, 96)
    rgb, d = w.render_inputs(0)
    tgt = _crop(w.targets[0], *crop)
    col, dep = gvs.gauss_splat(w.inputs, to_dev(d), to_dev(u32(rgb)), tgt)
    sf, se = gvs.fuse_depth_sphere(w.inputs, to_dev(d), tgt, w.z_near, w.z_far, w.mu)
    fused, _ = gvs.fuse_depth(w.inputs, to_dev(d), tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(w.inputs, to_dev(d), to_dev(u32(rgb)), tgt, fused=fused, mu_guide=w.mu)
    feats = gvs.blend_features(w.inputs, tgt, sp["warped_rgba"], sp["warped_depth"], sp["alpha"], fused)
    torch.cuda.synchronize()
    g = oracle_mod.gauss_splat(w.inputs, d, u32(rgb), tgt)
    ok = ~g["ambiguous"].astype(bool)
    assert np.all(np.abs(col.cpu().numpy() - g["color"]).max(axis=-1)[ok] <= 2e-5)
    s = oracle_mod.fuse_depth_sphere(w.inputs, d, tgt, w.z_near, w.z_far, w.mu)
    assert np.array_equal(sf.cpu().numpy().view(np.uint32), s["depth"].view(np.uint32))
    assert np.array_equal(se.cpu().numpy(), s["evals"])
    f = oracle_mod.blend_features(w.inputs, tgt, sp["warped_rgba"].cpu().numpy().view(np.uint32),
                                  sp["warped_depth"].cpu().numpy(), sp["alpha"].cpu().numpy(), fused.cpu().numpy())
    np.testing.assert_allclose(feats.cpu().numpy(), f, atol=2e-5, rtol=0)


def test_two_samples_per_ray(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(40, 30, 3, 2)
    _, d = w.render_inputs(0)
    fused, cross = gvs.fuse_depth(w.inputs, to_dev(d), w.targets[0], 2, w.z_near, w.z_far, w.mu)
    torch.cuda.synchronize()
    ref = oracle_mod.fuse_depth(w.inputs, d, w.targets[0], 2, w.z_near, w.z_far, w.mu)
    compare_fused(fused, cross, ref)


def test_thirty_two_views_everywhere(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(24, 18, 32, 64)
    rgb, d = w.render_inputs(0)
    tgt = w.targets[0]
    dd, cc = to_dev(d), to_dev(u32(rgb))
    sp = gvs.forward_splat(w.inputs, dd, cc, tgt)
    col, _ = gvs.gauss_splat(w.inputs, dd, cc, tgt)
    sf, _ = gvs.fuse_depth_sphere(w.inputs, dd, tgt, w.z_near, w.z_far, w.mu)
    torch.cuda.synchronize()
    rs = oracle_mod.forward_splat(w.inputs, d, u32(rgb), tgt)
    assert np.array_equal(sp["winner"].cpu().numpy(), rs["winner"])
    g = oracle_mod.gauss_splat(w.inputs, d, u32(rgb), tgt)
    ok = ~g["ambiguous"].astype(bool)
    assert np.all(np.abs(col.cpu().numpy() - g["color"]).max(axis=-1)[ok] <= 2e-5)
    s = oracle_mod.fuse_depth_sphere(w.inputs, d, tgt, w.z_near, w.z_far, w.mu)
    assert np.array_equal(sf.cpu().numpy().view(np.uint32), s["depth"].view(np.uint32))


def test_one_pixel_inputs(gvs, oracle_mod):
    """1x1 input views (the window is all border) into a small target."""
    from synth import Camera
    from synth import configs
    w = configs.tiny(40, 30, 3, 64)
    cams = [Camera(1, 1, c.fx, c.fy, 0.0, 0.0, c.R, c.t) for c in w.inputs]
    d = np.full((3, 1, 1), 2.0, np.float32)
    rgb = np.full((3, 1, 1), 0x00ff8040, np.uint32)
    tgt = w.targets[0]
    fused, cross = gvs.fuse_depth(cams, to_dev(d), tgt, 64, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(cams, to_dev(d), to_dev(rgb), tgt)
    torch.cuda.synchronize()
    ref = oracle_mod.fuse_depth(cams, d, tgt, 64, w.z_near, w.z_far, w.mu)
    compare_fused(fused, cross, ref)
    rs = oracle_mod.forward_splat(cams, d, rgb, tgt)
    assert np.array_equal(sp["winner"].cpu().numpy(), rs["winner"])
