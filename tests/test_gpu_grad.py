"""GPU adjoint of the fused depth (gvs_fuse_depth_backward) against the FP64 oracle adjoint.

Bar: per element |grad_gpu - grad_oracle| <= 1e-3 max|grad| + 1e-7 and cosine
similarity >= 0.9999 (FP32 atomics accumulate in varying order).  The
upstream gradient is zeroed on pixels the oracle flags as ambiguous, so both
sides differentiate the same crossing everywhere.
"""
import numpy as np
import pytest
import torch

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvs():
    assert torch.cuda.is_available()
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


def _check(ga, gr):
    scale = np.abs(gr).max()
    assert scale > 0
    err = np.abs(ga - gr)
    assert err.max() <= 1e-3 * scale + 1e-7, f"max err {err.max():.3e} vs scale {scale:.3e}"
    cos = float((ga * gr).sum() / (np.linalg.norm(ga) * np.linalg.norm(gr)))
    assert cos >= 0.9999, cos


def _case(gvs, oracle_mod, w, d, seed=0, window=7, half=False):
    tgt = w.targets[0]
    ref = oracle_mod.fuse_depth(w.inputs, d, tgt, w.num_samples, w.z_near, w.z_far, w.mu, window=window)
    G = np.random.default_rng(seed).standard_normal((tgt.height, tgt.width))
    G[ref["ambiguous"] == 1] = 0.0
    dd = torch.from_numpy(d.astype(np.float16) if half else d).cuda()
    N, H, W = d.shape
    ws = gvs.workspace(gvs.fuse_workspace_bytes(N, W, H))
    fused, cross = gvs.fuse_depth(w.inputs, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu, window=window, ws=ws)
    g = gvs.fuse_depth_backward(w.inputs, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu, ws, cross,
                                torch.from_numpy(G.astype(np.float32)).cuda(), window=window)
    torch.cuda.synchronize()
    assert np.array_equal(cross.cpu().numpy()[ref["ambiguous"] == 0], ref["index"][ref["ambiguous"] == 0])
    gr = oracle_mod.fuse_depth_grad(w.inputs, d, tgt, w.num_samples, w.z_near, w.z_far, w.mu, G, window=window)
    _check(g.cpu().numpy().astype(np.float64), gr)


def test_grad_tiny_ragged(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(70, 45, 3, 96)
    _, d = w.render_inputs(0)
    _case(gvs, oracle_mod, w, d)


@pytest.mark.parametrize("window", [1, 3, 9])
def test_grad_windows(gvs, oracle_mod, window):
    from synth import configs
    w = configs.tiny(40, 30, 2, 96)
    _, d = w.render_inputs(0)
    _case(gvs, oracle_mod, w, d, seed=window, window=window)


def test_grad_plain_320x240(gvs, oracle_mod):
    from synth import configs
    w = configs.plain_320x240()
    _, d = w.render_inputs(0)
    _case(gvs, oracle_mod, w, d, seed=4)


def test_grad_diff_640x360(gvs, oracle_mod):
    """The differentiable workload: 4 x 640x360, D = 96."""
    from synth import configs
    w = configs.diff_640x360()
    _, d = w.render_inputs(0)
    _case(gvs, oracle_mod, w, d, seed=5)


def test_grad_f16_depth(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(48, 36, 3, 96)
    _, d = w.render_inputs(0)
    _case(gvs, oracle_mod, w, d.astype(np.float16).astype(np.float32), seed=6, half=True)


@pytest.mark.parametrize("window", [7, 3])
def test_grad_half_map(gvs, oracle_mod, window):
    """The half2 map path of the adjoint, which re-sums nu from the depths instead of
    reading the weight from the map: against the FP32-map adjoint of the same FP16
    depths and against the oracle adjoint on those depths.  The forward's weights are
    rounded to half there (relative spacing 2^-11), which moves every weighted sum and
    so the gradient by about 1e-3 of its scale: the bar is 5e-3 of the scale per
    element and a cosine of at least 0.9995."""
    from synth import configs
    w = configs.tiny(56, 40, 3, 96)
    _, d = w.render_inputs(0)
    d16 = d.astype(np.float16)
    d32 = d16.astype(np.float32)
    tgt = w.targets[0]
    ref = oracle_mod.fuse_depth(w.inputs, d32, tgt, w.num_samples, w.z_near, w.z_far, w.mu, window=window)
    G = np.random.default_rng(window).standard_normal((tgt.height, tgt.width))
    G[ref["ambiguous"] == 1] = 0.0
    dd = torch.from_numpy(d16).cuda()
    N, H, W = d.shape
    Gt = torch.from_numpy(G.astype(np.float32)).cuda()
    grads = {}
    for half in (True, False):
        ws = gvs.workspace(gvs.fuse_workspace_bytes(N, W, H))
        fused, cross = gvs.fuse_depth(w.inputs, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu, window=window,
                                      ws=ws, map_half=half)
        g = gvs.fuse_depth_backward(w.inputs, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu, ws, cross, Gt,
                                    window=window, map_half=half)
        torch.cuda.synchronize()
        ok = ref["ambiguous"] == 0
        assert np.array_equal(cross.cpu().numpy()[ok], ref["index"][ok]), half
        grads[half] = g.cpu().numpy().astype(np.float64)
    gr = oracle_mod.fuse_depth_grad(w.inputs, d32, tgt, w.num_samples, w.z_near, w.z_far, w.mu, G, window=window)
    scale = np.abs(gr).max()
    assert scale > 0
    for a, b in ((grads[True], grads[False]), (grads[True], gr)):
        assert np.abs(a - b).max() <= 5e-3 * scale + 1e-7, np.abs(a - b).max() / scale
        cos = float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert cos >= 0.9995, cos
    _check(grads[False], gr)


def test_grad_identity_and_sum_rule(gvs):
    from synth import camera_at
    from synth.configs import arc_cameras
    cam = arc_cameras(40, 30, [7.0])[0]
    y, x = np.mgrid[0:30, 0:40]
    d = (2.0 + 0.4 * np.sin(x / 7.0) + 0.3 * np.cos(y / 5.0)).astype(np.float32)[None]
    G = np.random.default_rng(2).standard_normal((30, 40)).astype(np.float32)
    dd = torch.from_numpy(d).cuda()
    ws = gvs.workspace(gvs.fuse_workspace_bytes(1, 40, 30))
    f, c = gvs.fuse_depth([cam], dd, cam, 160, 0.5, 5.0, 0.05, ws=ws)
    g = gvs.fuse_depth_backward([cam], dd, cam, 160, 0.5, 5.0, 0.05, ws, c, torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    np.testing.assert_allclose(g.cpu().numpy()[0], G, rtol=1e-4, atol=1e-4)
    cams = [camera_at(48, 32, (x, y, 0.0)) for x, y in [(-0.05, 0.0), (0.05, 0.0), (0.0, 0.04)]]
    tgt = camera_at(48, 32, (0.01, 0.0, 0.0))
    dep = torch.full((3, 32, 48), 2.3, device="cuda")
    ws = gvs.workspace(gvs.fuse_workspace_bytes(3, 48, 32))
    f, c = gvs.fuse_depth(cams, dep, tgt, 256, 0.5, 5.0, 0.04, ws=ws)
    Gs = torch.zeros((32, 48), device="cuda")
    Gs[6:-6, 8:-8] = 1.0
    g = gvs.fuse_depth_backward(cams, dep, tgt, 256, 0.5, 5.0, 0.04, ws, c, Gs)
    torch.cuda.synchronize()
    assert abs(float(g.sum()) - float(Gs.sum())) <= 1e-4 * float(Gs.sum())


def test_autograd_function(gvs):
    from synth import configs
    w = configs.tiny(40, 30, 3, 96)
    _, d = w.render_inputs(0)
    dd = torch.from_numpy(d).cuda().requires_grad_(True)
    cfg = dict(num_samples=w.num_samples, z_near=w.z_near, z_far=w.z_far, mu=w.mu)
    fused, cross = gvs.FuseDepth.apply(dd, w.inputs, w.targets[0], cfg)
    r = torch.randn_like(fused)
    (fused * r).sum().backward()
    ws = gvs.workspace(gvs.fuse_workspace_bytes(*d.shape[:1], d.shape[2], d.shape[1]))
    f2, c2 = gvs.fuse_depth(w.inputs, dd.detach(), w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu, ws=ws)
    g2 = gvs.fuse_depth_backward(w.inputs, dd.detach(), w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu, ws, c2,
                                 r)
    torch.cuda.synchronize()
    assert torch.equal(fused, f2)
    assert torch.allclose(dd.grad, g2, rtol=1e-5, atol=1e-6)
