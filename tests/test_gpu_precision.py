"""Reduced-precision storage: FP16 depth and half2 (depth, weight) maps, FP32 arithmetic.

(i) Against the FP64 oracle run on the FP16-rounded depths, the kernel's own
    arithmetic must meet the FP32 bar: bit-exact integer maps and copies,
    fused depth within 1e-4 relative on non-ambiguous pixels.
(ii) Against the oracle on the original FP32 depths the total error (storage
    rounding included) is reported, and only bounded loosely here: FP16 has an
    ulp of 3.9 mm on [4, 8) m.
"""
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


def _half(a):
    return np.asarray(a, np.float32).astype(np.float16)


def test_refine_f16_copies_bits(gvs, oracle_mod):
    rng = np.random.default_rng(5)
    N, H, W = 3, 29, 41
    a = rng.integers(0, 256, (N, H, W, 4), dtype=np.uint8)
    b = np.clip(a.astype(int) + rng.integers(-10, 11, a.shape), 0, 255).astype(np.uint8)
    d = _half(rng.uniform(0.5, 9.0, (N, H, W)))
    prev = _half(rng.uniform(0.5, 9.0, (N, H, W)))
    ref_s, ref_m = oracle_mod.refine_depth(a, b, d.astype(np.float32), prev.astype(np.float32), 0.03)
    st = torch.from_numpy(prev.copy()).cuda()
    mask = torch.empty((N, H, W), dtype=torch.uint8, device="cuda")
    gvs.refine_depth(to_dev(u32(a)), to_dev(u32(b)), torch.from_numpy(d).cuda(), st, mask, tau=0.03)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy(), ref_m)
    assert np.array_equal(st.cpu().numpy().astype(np.float32).view(np.uint32), ref_s.view(np.uint32))


@pytest.mark.parametrize("depth_half,map_half", [(True, True), (True, False), (False, True)])
def test_fuse_half_storage_plain(gvs, oracle_mod, depth_half, map_half):
    from synth import configs
    w = configs.plain_320x240()
    _, d = w.render_inputs(0)
    d16 = _half(d)
    d_in = torch.from_numpy(d16).cuda() if depth_half else torch.from_numpy(d).cuda()
    fused, cross = gvs.fuse_depth(w.inputs, d_in, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu,
                                  map_half=map_half)
    torch.cuda.synchronize()
    # the map (or the input) holds FP16 depths: the oracle gets the same rounded values
    ref = oracle_mod.fuse_depth(w.inputs, d16.astype(np.float32), w.targets[0], w.num_samples, w.z_near, w.z_far,
                                w.mu)
    compare_fused(fused, cross, ref)
    # (ii) total error against the unrounded inputs, over pixels where both find the same crossing
    full = oracle_mod.fuse_depth(w.inputs, d, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu)
    g = fused.cpu().numpy().astype(np.float64)
    same = (cross.cpu().numpy() == full["index"]) & (full["index"] >= 0)
    rel = np.abs(g[same] - full["depth"][same]) / full["depth"][same]
    print(f"total error vs FP32 inputs: median {np.median(rel):.2e}, p99 {np.percentile(rel, 99):.2e}")
    assert np.median(rel) < 2e-3


def test_fuse_half_storage_full_size_sampled(gvs, oracle_mod):
    from synth import configs
    w = configs.mixed_16x1080p()
    _, d = w.render_inputs(3)
    d16 = _half(d)
    tgt = w.targets[0]
    fused, cross = gvs.fuse_depth(w.inputs, torch.from_numpy(d16).cuda(), tgt, w.num_samples, w.z_near, w.z_far,
                                  w.mu, map_half=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    pix = np.stack([rng.integers(0, tgt.width, 1024), rng.integers(0, tgt.height, 1024)], 1).astype(np.int32)
    ref = oracle_mod.fuse_depth(w.inputs, d16.astype(np.float32), tgt, w.num_samples, w.z_near, w.z_far, w.mu,
                                pixels=pix)
    compare_fused(fused, cross, ref, (pix[:, 1], pix[:, 0]))


def test_weight_map_half(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(37, 29, 2, 16)
    _, d = w.render_inputs(0)
    d16 = _half(d)
    m = gvs.weight_map(torch.from_numpy(d16).cuda(), w.mu, map_half=True)
    torch.cuda.synchronize()
    mp = m[: d.size * 4].view(torch.float16).cpu().numpy().astype(np.float32).reshape(d.shape + (2,))
    for k in range(d.shape[0]):
        for v in range(0, d.shape[1], 3):
            for u in range(0, d.shape[2], 2):
                ref = oracle_mod.weight(d16[k].astype(np.float32), u, v, w.mu)
                assert abs(mp[k, v, u, 1] - ref) <= 2.0 ** -10 * ref + 1e-6, (k, v, u)
                assert mp[k, v, u, 0] == d16[k, v, u].astype(np.float32)


def test_splat_f16_depth_bit_exact(gvs, oracle_mod):
    from synth import configs
    w = configs.headline_8x1080p()
    rgb, d = w.render_inputs(2)
    d16 = _half(d)
    tgt = w.targets[0]
    _, gt = w.render_target_gt(tgt, 2)
    out = gvs.forward_splat(w.inputs, torch.from_numpy(d16).cuda(), to_dev(u32(rgb)), tgt,
                            fused=to_dev(gt.astype(np.float32)), mu_guide=w.mu)
    torch.cuda.synchronize()
    ref = oracle_mod.forward_splat(w.inputs, d16.astype(np.float32), u32(rgb), tgt, mu_guide=w.mu,
                                   fused=gt.astype(np.float32).astype(np.float64))
    for k in ["winner", "alpha", "guided"]:
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
    assert np.array_equal(out["warped_rgba"].cpu().numpy().view(np.uint32), ref["warped_rgba"])
    assert np.array_equal(out["warped_depth"].cpu().numpy().view(np.uint32), ref["warped_depth"].view(np.uint32))
