"""GPU parity of the blending-network input and the Eq. 4-5 blend against the
FP64 oracle, on the outputs of the GPU splat and fusion (both sides get the
same arrays).  Copies (depths, alphas, TSDF depth) are exact; colours and
camera maps within 1e-6; the normal and ray dot products within 2e-5; the
blended image within 1e-5 and L_Depth within 1e-5 relative."""
import numpy as np
import pytest
import torch

from gpu_util import to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvs():
    assert torch.cuda.is_available()
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


def _frame(gvs, w, K=None):
    rgb, d = w.render_inputs(0)
    cams = w.inputs if K is None else w.inputs[:K]
    dd, cc = to_dev(d[:len(cams)]), to_dev(u32(rgb)[:len(cams)])
    tgt = w.targets[0]
    fused, _ = gvs.fuse_depth(cams, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(cams, dd, cc, tgt, fused=fused, mu_guide=w.mu)
    torch.cuda.synchronize()
    return cams, tgt, sp, fused


def _features_case(gvs, oracle_mod, w):
    cams, tgt, sp, fused = _frame(gvs, w)
    K = len(cams)
    f = gvs.blend_features(cams, tgt, sp["warped_rgba"], sp["warped_depth"], sp["alpha"], fused)
    torch.cuda.synchronize()
    got = f.cpu().numpy().astype(np.float64)
    ref = oracle_mod.blend_features(cams, tgt, sp["warped_rgba"].cpu().numpy().view(np.uint32),
                                    sp["warped_depth"].cpu().numpy(), sp["alpha"].cpu().numpy(),
                                    fused.cpu().numpy())
    np.testing.assert_allclose(got[:3 * K], ref[:3 * K], atol=1e-6, rtol=0)
    assert np.array_equal(got[3 * K:5 * K + 1], ref[3 * K:5 * K + 1])
    np.testing.assert_allclose(got[5 * K + 1:7 * K + 1], ref[5 * K + 1:7 * K + 1], atol=2e-5, rtol=0)
    np.testing.assert_allclose(got[7 * K + 1:], ref[7 * K + 1:], atol=1e-6, rtol=0)
    # the geometry channels are not trivially zero
    assert (np.abs(ref[5 * K + 1:6 * K + 1]) > 0.1).mean() > 0.2
    return f, (cams, tgt, sp, fused)


def test_features_tiny(gvs, oracle_mod):
    from synth import configs
    _features_case(gvs, oracle_mod, configs.tiny(70, 45, 3, 96))


def test_features_plain_320x240(gvs, oracle_mod):
    from synth import configs
    _features_case(gvs, oracle_mod, configs.plain_320x240())


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_features_half_storage_rounds_fp32(gvs, oracle_mod, dtype):
    """Half-precision planes are the FP32 values rounded to nearest."""
    from synth import configs
    f32, (cams, tgt, sp, fused) = _features_case(gvs, oracle_mod, configs.tiny(70, 45, 3, 96))
    fh = gvs.blend_features(cams, tgt, sp["warped_rgba"], sp["warped_depth"], sp["alpha"], fused, dtype=dtype)
    torch.cuda.synchronize()
    assert torch.equal(fh, f32.to(dtype))


@pytest.mark.parametrize("wdtype", [torch.float32, torch.bfloat16])
def test_blend_matches_oracle(gvs, oracle_mod, wdtype):
    from synth import configs
    w = configs.plain_320x240()
    cams, tgt, sp, fused = _frame(gvs, w)
    K = len(cams)
    g = torch.Generator(device="cuda").manual_seed(3)
    net = torch.rand((K + 4, tgt.height, tgt.width), generator=g, device="cuda").to(wdtype)
    wk, wbg, ibg = net[:K], net[K], net[K + 1:]
    img, L = gvs.blend(sp["warped_rgba"], sp["alpha"], sp["warped_depth"], fused, wk, wbg, ibg)
    img2, L2 = gvs.blend(sp["warped_rgba"], sp["alpha"], sp["warped_depth"], fused, wk, wbg, ibg)
    torch.cuda.synchronize()
    assert torch.equal(img, img2) and torch.equal(L, L2)     # fixed-order reduction
    n64 = net.double().cpu().numpy()
    ref, Lr = oracle_mod.blend(sp["warped_rgba"].cpu().numpy().view(np.uint32), sp["alpha"].cpu().numpy(),
                               sp["warped_depth"].cpu().numpy(), fused.cpu().numpy(), n64[:K], n64[K], n64[K + 1:])
    np.testing.assert_allclose(img.cpu().numpy(), ref, atol=1e-5, rtol=0)
    assert L.item() == pytest.approx(Lr, rel=1e-5)


def test_network_path_runs(gvs):
    """Features -> random-weight U-Net (cuDNN, bf16) -> blend on the 4 views closest to the
    target: finite outputs of the right shapes (an end-to-end timing path, not a parity test)."""
    from paper_2505_18932_gb300.blendnet import BlendUNet
    from synth import configs
    w = configs.tiny(96, 64, 6, 64)
    sel = gvs.select_views(w.inputs, w.targets[0], 4)
    rgb, d = w.render_inputs(0)
    cams = [w.inputs[i] for i in sel]
    dd, cc = to_dev(d[sel]), to_dev(u32(rgb)[sel])
    tgt = w.targets[0]
    fused, _ = gvs.fuse_depth(cams, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(cams, dd, cc, tgt, fused=fused, mu_guide=w.mu)
    feats = gvs.blend_features(cams, tgt, sp["warped_rgba"], sp["warped_depth"], sp["alpha"], fused,
                               dtype=torch.bfloat16)
    net = BlendUNet(4).cuda().to(torch.bfloat16).eval()
    with torch.no_grad():
        wk, wbg, ibg = net(feats[None])
    img, L = gvs.blend(sp["warped_rgba"], sp["alpha"], sp["warped_depth"], fused, wk, wbg, ibg)
    torch.cuda.synchronize()
    assert feats.shape == (37, 64, 96) and img.shape == (3, 64, 96)
    assert torch.isfinite(img).all() and np.isfinite(L.item())
