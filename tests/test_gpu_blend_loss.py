"""The uniform-blend training loss (Sec. 3.3's w_l1 L1 + w_depth L_Depth on Eq. 4 with
unit weights) and the differentiable splat's adjoint fed by its per-pixel gradient.

* gvs_uniform_blend_loss against the FP64 oracle on seeded inputs: the three losses within
  1e-5 relative, the per-pixel gradients within 1e-6 relative where the signs they carry are
  decided away from 0 (|B - GT| and |F - Dbar| above 1e-5) and exactly 0 at exact ties and at
  uncovered pixels.
* gvs_soft_splat_backward_blended equals gvs_soft_splat_backward fed with the same gradient
  spread to every covering view, bit for bit (the same arithmetic per term).
* gvs_uniform_blend_loss_grad, run later on the loss call's workspace, gives the loss call's
  gradients bit for bit, and times an upstream scalar read on the device, the same values as
  multiplying them afterwards; the loss itself is bit-reproducible.
* SoftSplatBlendLoss gives the gradients of the library calls it wires together, and its
  loss equals the same step written with torch operations on the splat's outputs.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvs():
    assert torch.cuda.is_available()
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


@pytest.mark.parametrize("shape", [(4, 37, 53), (8, 360, 640), (1, 16, 16)])
def test_loss_matches_oracle(gvs, oracle_mod, shape):
    K, H, W = shape
    rng = np.random.default_rng(K * 100 + H)
    color = rng.random((K, H, W, 4)).astype(np.float32)
    alpha = (rng.random((K, H, W)) < 0.6).astype(np.uint8)
    color[alpha == 0] = 0.0
    wd = (rng.random((K, H, W)) * 4 + 1).astype(np.float32) * alpha
    fused = (rng.random((H, W)) * 4 + 1).astype(np.float32)
    fused[rng.random((H, W)) < 0.1] = 0.0
    gt = rng.random((H, W, 3)).astype(np.float32)
    # exact ties, as flat colour regions give them: every covering view equals the ground
    # truth (and the fused depth equals every warped depth) on a tenth of the pixels
    tie = rng.random((H, W)) < 0.1
    for k in range(K):
        m = tie & (alpha[k] > 0)
        color[k][m, :3] = gt[m]
        wd[k][m] = fused[m]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, gp, gf = gvs.uniform_blend_loss(dev(color), dev(alpha), dev(wd), dev(fused), dev(gt))
    torch.cuda.synchronize()
    L, L1, LD, g = oracle_mod.uniform_blend_loss(color, alpha, wd, fused, gt)
    got = loss.cpu().numpy()
    for a, b in zip(got, (L, L1, LD)):
        assert abs(a - b) <= 1e-5 * max(abs(b), 1e-12), (got, (L, L1, LD))
    gp, gf = gp.cpu().numpy().astype(np.float64), gf.cpu().numpy().astype(np.float64)
    A = alpha.sum(0)
    B = (alpha[..., None] * color[..., :3].astype(np.float64)).sum(0) / np.maximum(A, 1)[..., None]
    Dbar = (alpha * wd.astype(np.float64)).sum(0) / np.maximum(A, 1)
    # compared everywhere except where B - GT or F - Dbar is nonzero but below 1e-5 (a sign an
    # FP32 sum could still decide otherwise); exact ties must give exactly 0, as in FP64
    clear_rgb = (np.abs(B - gt) > 1e-5) | (B == gt)
    clear_d = (np.abs(fused - Dbar) > 1e-5) | (fused == Dbar)
    ok = clear_rgb & (A > 0)[..., None]
    assert np.allclose(gp[..., :3][ok], g["rgb"][ok], rtol=1e-6, atol=0)
    okd = clear_d & (A > 0)
    assert np.allclose(gp[..., 3][okd], g["depth"][okd], rtol=1e-6, atol=0)
    assert np.allclose(gf[okd], g["fused"][okd], rtol=1e-6, atol=0)
    assert (gp[A == 0] == 0).all() and (gf[A == 0] == 0).all()
    tied = tie & (A > 0)
    assert tied.sum() > 0 and (gp[tied][:, :3] == 0).all()
    assert (gp[tied & (fused > 0)][:, 3] == 0).all() and (gf[tied] == 0).all()
    # the comparisons above cover nearly every pixel where the terms exist
    assert clear_rgb[A > 0].mean() > 0.99 and clear_d[(A > 0) & (fused > 0)].mean() > 0.99


@pytest.mark.parametrize("shape", [(8, 360, 640), (3, 17, 29)])
def test_grad_stage_on_kept_workspace(gvs, shape):
    K, H, W = shape
    rng = np.random.default_rng(7 + K)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    alpha = (rng.random((K, H, W)) < 0.7).astype(np.uint8)
    color = rng.random((K, H, W, 4)).astype(np.float32) * alpha[..., None]
    wd = (rng.random((K, H, W)) * 3 + 1).astype(np.float32) * alpha
    fused = (rng.random((H, W)) * 3 + 1).astype(np.float32)
    gt = rng.random((H, W, 3)).astype(np.float32)
    args = (dev(color), dev(alpha), dev(wd), dev(fused), dev(gt))
    ws = gvs.workspace(gvs.blend_loss_workspace_bytes(H, W), "cuda")
    loss, gp, gf = gvs.uniform_blend_loss(*args, ws=ws)
    loss2, _, _ = gvs.uniform_blend_loss(*args, want_grad=False)
    g1, f1 = gvs.uniform_blend_loss_grad(ws, H, W)
    torch.cuda.synchronize()
    assert torch.equal(loss, loss2)  # the fixed-order reduction
    assert torch.equal(g1, gp) and torch.equal(f1, gf)
    assert gp.abs().sum() > 0 and gf.abs().sum() > 0
    for u in (2.5, -0.3, 0.0):
        gu = torch.tensor(u, dtype=torch.float32, device="cuda")
        g2, f2 = gvs.uniform_blend_loss_grad(ws, H, W, gu)
        torch.cuda.synchronize()
        assert torch.equal(g2, gp * gu) and torch.equal(f2, gf * gu), u


def test_each_gradient_output_alone(gvs):
    """Through the C ABI: either gradient output may be NULL, in the loss call and in the
    gradient stage, and the other comes out as when both are asked for."""
    lib = gvs.load()
    K, H, W = 3, 24, 40
    rng = np.random.default_rng(12)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    alpha = (rng.random((K, H, W)) < 0.7).astype(np.uint8)
    color = dev(rng.random((K, H, W, 4)).astype(np.float32) * alpha[..., None])
    wd = dev((rng.random((K, H, W)) * 3 + 1).astype(np.float32) * alpha)
    fused = dev((rng.random((H, W)) * 3 + 1).astype(np.float32))
    gt = dev(rng.random((H, W, 3)).astype(np.float32))
    alpha = dev(alpha)
    loss, gp, gf = gvs.uniform_blend_loss(color, alpha, wd, fused, gt)
    P = gvs._ptr
    for want_pixel in (True, False):
        ws = gvs.workspace(gvs.blend_loss_workspace_bytes(H, W), "cuda")
        l2 = torch.empty(3, dtype=torch.float64, device="cuda")
        gp2 = torch.zeros((H, W, 4), device="cuda") if want_pixel else None
        gf2 = None if want_pixel else torch.zeros((H, W), device="cuda")
        st = lib.gvs_uniform_blend_loss(K, W, H, P(color), P(alpha), P(wd), P(fused), P(gt), 0.8, 0.1, P(l2),
                                        P(gp2), P(gf2), P(ws), ws.numel(), None)
        assert st == 0
        gp3 = torch.zeros((H, W, 4), device="cuda") if want_pixel else None
        gf3 = None if want_pixel else torch.zeros((H, W), device="cuda")
        st = lib.gvs_uniform_blend_loss_grad(W, H, None, P(gp3), P(gf3), P(ws), ws.numel(), None)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.equal(l2, loss)
        if want_pixel:
            assert torch.equal(gp2, gp) and torch.equal(gp3, gp)
        else:
            assert torch.equal(gf2, gf) and torch.equal(gf3, gf)


def _soft_case(gvs, name="diff_640x360"):
    from synth import configs
    w = getattr(configs, name)()
    rgb, d = w.render_inputs(0)
    tgt = w.targets[0]
    depth = torch.from_numpy(d).cuda()
    color = torch.from_numpy(np.asarray(rgb, np.float32) / 255.0).cuda()
    fwd = gvs.soft_splat(w.inputs, depth, color, tgt, mu_band=w.mu)
    gt_rgb, _ = w.render_target_gt(tgt, 0)
    gt = torch.from_numpy(np.ascontiguousarray(gt_rgb[..., :3], np.float32) / 255.0).cuda()
    return w, tgt, depth, color, fwd, gt


def test_blended_adjoint_equals_per_view_adjoint(gvs):
    w, tgt, depth, color, fwd, gt = _soft_case(gvs)
    rng = np.random.default_rng(4)
    gp = torch.from_numpy(rng.standard_normal((tgt.height, tgt.width, 4)).astype(np.float32)).cuda()
    a = fwd["alpha"].float()
    gd1, gc1 = gvs.soft_splat_backward_blended(w.inputs, depth, color, tgt, fwd, gp, mu_band=w.mu)
    gcol = (a[..., None] * gp[None]).contiguous()
    gc_per = gcol.clone()
    gc_per[..., 3] = 0.0
    gd2, gc2 = gvs.soft_splat_backward(w.inputs, depth, color, tgt, fwd, gc_per, (a * gp[None, ..., 3]).contiguous(),
                                       mu_band=w.mu)
    torch.cuda.synchronize()
    assert torch.equal(gd1, gd2) and torch.equal(gc1, gc2)
    assert gd1.abs().sum() > 0 and gc1.abs().sum() > 0


def test_autograd_function(gvs):
    """SoftSplatBlendLoss's gradients are those of the library calls it wires together, and
    its loss is the one the same step written in torch operations computes
    (the gradients of that step differ where a blended value ties the ground truth: its
    FP32 sums resolve the tie differently from the FP64 definition the library follows)."""
    w, tgt, depth, color, _, gt = _soft_case(gvs)
    N = len(w.inputs)
    fused, _ = gvs.fuse_depth(w.inputs, depth, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    cfg = {"mu_band": w.mu}
    d1, c1, f1 = (t.detach().clone().requires_grad_(True) for t in (depth, color, fused))
    L1 = gvs.SoftSplatBlendLoss.apply(d1, c1, f1, w.inputs, tgt, gt, cfg)
    L1.backward()
    # the same calls by hand
    fwd = gvs.soft_splat(w.inputs, depth, color, tgt, mu_band=w.mu)
    loss, gp, gf = gvs.uniform_blend_loss(fwd["color"], fwd["alpha"], fwd["depth"], fused, gt)
    gd, gc = gvs.soft_splat_backward_blended(w.inputs, depth, color, tgt, fwd, gp, mu_band=w.mu)
    torch.cuda.synchronize()
    # the splat accumulates its colours with float atomics, so two forward calls agree to the
    # last bits, not bit for bit, and the many exact ties of these scenes (flat colour: the
    # blend equals the ground truth) can be met by one call and missed by the other, which
    # moves the L1 subgradient there between 0 and its full value
    assert abs(float(L1.detach()) - float(loss[0])) <= 1e-6 * float(loss[0])
    for a, b in ((d1.grad, gd), (c1.grad, gc), (f1.grad, gf)):
        cos = torch.nn.functional.cosine_similarity(a.flatten().double(), b.flatten().double(), dim=0)
        assert cos > 0.999, float(cos)
        off = (a - b).abs() > 1e-4 * b.abs().max() + 1e-12
        assert off.float().mean() < 1e-2, (int(off.sum()), off.numel())
    assert gd.abs().sum() > 0 and gc.abs().sum() > 0 and gf.abs().sum() > 0
    # the loss of the same step in torch operations on the splat's outputs
    col, wdep, alpha = fwd["color"], fwd["depth"], fwd["alpha"]
    asum = alpha.sum(0, dtype=torch.float32)
    valid = asum > 0
    inv = 1.0 / asum.clamp_min(1.0)
    blend = col.sum(0)[..., :3] * inv.unsqueeze(-1)
    l1 = ((blend - gt).abs().sum(-1) * valid).sum() / (3.0 * valid.sum().clamp_min(1))
    dblend = wdep.sum(0) * inv
    dvalid = valid & (fused > 0)
    ld = ((fused - dblend).abs() * dvalid).sum() / (N * dvalid.numel())
    L2 = float(0.8 * l1 + 0.1 * ld)
    assert abs(float(loss[0]) - L2) <= 1e-5 * abs(L2)
