"""Full-size parity against the FP64 oracle, in the launch configurations the
benchmark times:

* the confidence-weight map of all 8 views at 1920x1080 (FP32 and half2 maps)
  against the Supplement A.1 weight evaluated by the oracle, at 4096 seeded
  pixels per view: a quarter on the image border, a quarter next to planted
  invalid depths, the rest anywhere;
* the fused depth of the 8 x 1080p frame at 16384 target pixels, stratified:
  the target border, pixels whose analytic surface puts a sample inside the
  truncation band in front of it (where a crossing is expected), and the rest;
* the batched serving plan (8 x 1280x720 inputs, 16 targets of four sizes,
  2 frames, one CUDA graph): refined state bit for bit, fused depth at seeded
  pixels of every (frame, target) item, and the splat of one target of each
  size per frame (winner, colour, depth bits and alpha bit for bit; the guided
  mask where the oracle's own fused depth is known).
"""
import numpy as np
import pytest
import torch

from gpu_util import compare_fused, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


def _plant_invalid(d, rng):
    """Invalid depths (NaN, 0, -1, inf) in small patches, two of them touching the border."""
    N, H, W = d.shape
    sites = []
    for k in range(N):
        for n, bad in enumerate([np.nan, 0.0, -1.0, np.inf, np.nan, 0.0]):
            if n == 0:
                y, x = 0, int(rng.integers(0, W - 3))
            elif n == 1:
                y, x = int(rng.integers(0, H - 3)), W - 2
            else:
                y, x = int(rng.integers(3, H - 6)), int(rng.integers(3, W - 6))
            h, w = int(rng.integers(1, 4)), int(rng.integers(1, 4))
            d[k, y:y + h, x:x + w] = bad
            sites.append((k, y, x))
    return sites


def _map_pixels(shape, sites, rng, n=4096):
    """Per view n pixels: n/4 on the border (within 3 px), n/4 within 4 px of a planted
    invalid patch, n/2 uniform."""
    N, H, W = shape
    out = []
    for k in range(N):
        q = n // 4
        side = rng.integers(0, 4, q)
        a = rng.integers(0, 4, q)
        bx = np.where(side == 0, a, np.where(side == 1, W - 1 - a, rng.integers(0, W, q)))
        by = np.where(side == 2, a, np.where(side == 3, H - 1 - a, rng.integers(0, H, q)))
        near = [s for s in sites if s[0] == k]
        pick = rng.integers(0, len(near), q)
        nx = np.clip(np.array([near[i][2] for i in pick]) + rng.integers(-4, 8, q), 0, W - 1)
        ny = np.clip(np.array([near[i][1] for i in pick]) + rng.integers(-4, 8, q), 0, H - 1)
        ux, uy = rng.integers(0, W, n - 2 * q), rng.integers(0, H, n - 2 * q)
        out.append((np.concatenate([bx, nx, ux]), np.concatenate([by, ny, uy])))
    return out


@pytest.mark.parametrize("map_half", [False, True])
def test_weight_map_full_size_matches_oracle(gvs, oracle_mod, map_half):
    from synth import configs
    w = configs.headline_8x1080p()
    _, d = w.render_inputs(1)
    rng = np.random.default_rng(21)
    sites = _plant_invalid(d, rng)
    m = gvs.weight_map(to_dev(d), w.mu, map_half=map_half)
    torch.cuda.synchronize()
    if map_half:
        mp = m[: d.size * 4].view(torch.float16).cpu().numpy().astype(np.float32).reshape(d.shape + (2,))
        # the half2 map stores the depth rounded to half and takes the weight over those depths
        ds = d.astype(np.float16).astype(np.float32)
    else:
        mp = m[: d.size * 8].view(torch.float32).cpu().numpy().reshape(d.shape + (2,))
        ds = d
    checked = invalid_centre = invalid_near = 0
    for k, (xs, ys) in enumerate(_map_pixels(d.shape, sites, rng)):
        view = np.ascontiguousarray(ds[k])
        for u, v in zip(xs.tolist(), ys.tolist()):
            ref = oracle_mod.weight(view, u, v, w.mu)
            got = float(mp[k, v, u, 1])
            if map_half:
                assert abs(got - ref) <= 2.0 ** -10 * ref + 1e-6, (k, v, u, got, ref)
            else:
                assert abs(got - ref) <= 2e-6 * max(ref, 1e-3), (k, v, u, got, ref)
            dv = view[v, u]
            ok = np.isfinite(dv) and dv > 0
            assert mp[k, v, u, 0] == (dv if ok else 0.0), (k, v, u)
            checked += 1
            invalid_centre += not ok
            win = view[max(v - 3, 0):v + 4, max(u - 3, 0):u + 4]
            invalid_near += ok and not (np.isfinite(win) & (win > 0)).all()
    assert checked == 8 * 4096
    assert invalid_centre > 100 and invalid_near > 500, (invalid_centre, invalid_near)


def _crossing_candidates(w, tgt, frame, rng, n):
    """Target pixels whose analytic first-hit depth d has a sample z_s in (d, d + mu): there
    the uniform march is expected to report a crossing.  From the scene generator only."""
    _, gt = w.render_target_gt(tgt, frame)
    dz = (w.z_far - w.z_near) / (w.num_samples - 1)
    s = np.ceil((gt - w.z_near) / dz)
    zs = w.z_near + s * dz
    ok = np.isfinite(gt) & (gt > w.z_near) & (zs > gt) & (zs < gt + w.mu) & (s < w.num_samples)
    ys, xs = np.nonzero(ok)
    pick = rng.choice(len(xs), size=min(n, len(xs)), replace=False)
    return xs[pick], ys[pick]


def test_fuse_full_size_stratified(gvs, oracle_mod):
    """16384 target pixels of the 8 x 1080p frame: 4096 on the border (within 4 px),
    8192 expected crossings, 4096 anywhere."""
    from synth import configs
    w = configs.headline_8x1080p()
    _, d = w.render_inputs(1)
    tgt = w.targets_at(1)[0]
    Wt, Ht = tgt.width, tgt.height
    rng = np.random.default_rng(33)
    q = 4096
    side = rng.integers(0, 4, q)
    a = rng.integers(0, 4, q)
    bx = np.where(side == 0, a, np.where(side == 1, Wt - 1 - a, rng.integers(0, Wt, q)))
    by = np.where(side == 2, a, np.where(side == 3, Ht - 1 - a, rng.integers(0, Ht, q)))
    cx, cy = _crossing_candidates(w, tgt, 1, rng, 2 * q)
    ux, uy = rng.integers(0, Wt, q), rng.integers(0, Ht, q)
    pix = np.stack([np.concatenate([bx, cx, ux]), np.concatenate([by, cy, uy])], 1).astype(np.int32)
    assert len(pix) == 4 * q
    fused, cross = gvs.fuse_depth(w.inputs, to_dev(d), tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    torch.cuda.synchronize()
    ref = oracle_mod.fuse_depth(w.inputs, d, tgt, w.num_samples, w.z_near, w.z_far, w.mu, pixels=pix)
    compare_fused(fused, cross, ref, (pix[:, 1], pix[:, 0]))
    found = ref["index"][q:3 * q] >= 0
    assert found.mean() > 0.9, found.mean()


def test_batched_plan_matches_oracle(gvs, oracle_mod):
    from paper_2505_18932_gb300 import batch
    from synth import configs
    w = configs.batched_16_targets()
    fr = [w.render_inputs(t) for t in (0, 1, 2)]
    rgba = [to_dev(u32(r)) for r, _ in fr]
    dep = [to_dev(d) for _, d in fr]
    plan = batch.BatchPlan(w.inputs, w.targets, rgba[1:], dep[1:], w.num_samples, w.z_near, w.z_far, w.mu,
                           tau=w.tau, rgba_prev=rgba[0], state0=dep[0], variant=None, graph=True)
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(44)
    state = fr[0][1]
    seen_sizes = set()
    for f in range(2):
        rgb_t, d_t = fr[f + 1]
        rgb_p = fr[f][0]
        state, _ = oracle_mod.refine_depth(rgb_t, rgb_p, d_t, state, w.tau)
        assert np.array_equal(plan.states[f].cpu().numpy().view(np.uint32), state.view(np.uint32)), f
        for n, tgt in enumerate(w.targets):
            Wt, Ht = tgt.width, tgt.height
            q = 64
            side = rng.integers(0, 4, q)
            a = rng.integers(0, 3, q)
            bx = np.where(side == 0, a, np.where(side == 1, Wt - 1 - a, rng.integers(0, Wt, q)))
            by = np.where(side == 2, a, np.where(side == 3, Ht - 1 - a, rng.integers(0, Ht, q)))
            cx, cy = _crossing_candidates(w, tgt, f + 1, rng, 128)
            ux, uy = rng.integers(0, Wt, q), rng.integers(0, Ht, q)
            pix = np.stack([np.concatenate([bx, cx, ux]), np.concatenate([by, cy, uy])], 1).astype(np.int32)
            rf = oracle_mod.fuse_depth(w.inputs, state, tgt, w.num_samples, w.z_near, w.z_far, w.mu, pixels=pix)
            where = (pix[:, 1], pix[:, 0])
            compare_fused(plan.fused[f][n], plan.cross[f][n], rf, where)
            if (Wt, Ht) in seen_sizes and n != len(w.targets) - 1:
                continue
            seen_sizes.add((Wt, Ht))
            # the splat of this item: the guided mask takes the oracle's fused depth at the
            # sampled pixels (0 elsewhere) and is compared there, off the flagged pixels
            fused_ref = np.zeros((Ht, Wt))
            fused_ref[where] = rf["depth"]
            ref = oracle_mod.forward_splat(w.inputs, state, u32(rgb_t), tgt, mu_guide=w.mu, fused=fused_ref)
            out = plan.splat[f][n]
            assert np.array_equal(out["winner"].cpu().numpy(), ref["winner"]), (f, n)
            assert np.array_equal(out["warped_rgba"].cpu().numpy().view(np.uint32), ref["warped_rgba"]), (f, n)
            assert np.array_equal(out["warped_depth"].cpu().numpy().view(np.uint32),
                                  ref["warped_depth"].view(np.uint32)), (f, n)
            assert np.array_equal(out["alpha"].cpu().numpy(), ref["alpha"]), (f, n)
            g = out["guided"].cpu().numpy()[:, where[0], where[1]]
            amb = ref["guided_ambiguous"].astype(bool)[:, where[0], where[1]] | \
                rf["ambiguous"].astype(bool)[None]
            assert np.array_equal(g[~amb], ref["guided"][:, where[0], where[1]][~amb]), (f, n)
    assert len(seen_sizes) == 4
