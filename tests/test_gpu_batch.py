"""Batched serving path: every march variant gives the same bits; the persistent
batched fusion equals one fusion per item; the CUDA-graph plan equals the same
calls made eagerly and the single-view API; the autotuner records its choice."""
import json
import os

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


def _targets(w):
    from synth import camera_at
    return [camera_at(48, 32, (0.05, 0.01, -2.0)), camera_at(70, 45, (0.0, 0.0, -2.0)),
            camera_at(64, 48, (-0.04, -0.02, -2.0))]


@pytest.mark.parametrize("K", [5, 8, 12, 16, 32])
def test_variants_bit_identical(gvs, K):
    """Every variant, the lane-per-ray bundle shapes and the warp-per-ray mapping, gives
    the default's fused depth and crossing index bit for bit (K = 5 and 12 run the
    per-view-guarded 8- and 16-view kernels, 32 the 32-view ones)."""
    from synth import configs
    w = configs.tiny(70, 45, K, 96)
    _, d = w.render_inputs(0)
    dd = to_dev(d)
    ref = None
    for v in range(7):
        f, c = gvs.fuse_depth(w.inputs, dd, w.targets[0], w.num_samples, w.z_near, w.z_far, w.mu, variant=v)
        torch.cuda.synchronize()
        if ref is None:
            ref = (f.clone(), c.clone())
            assert (c >= 0).float().mean() > 0.5
        else:
            assert torch.equal(f.view(torch.int32), ref[0].view(torch.int32)) and torch.equal(c, ref[1]), v


def test_batched_equals_per_item(gvs):
    from synth import configs
    w = configs.tiny(64, 48, 8, 96)
    tg = _targets(w)
    maps = []
    for fr in range(2):
        _, d = w.render_inputs(fr)
        maps.append(gvs.weight_map(to_dev(d), w.mu))
    refs = [[gvs.fuse_depth_from_map(w.inputs, m, (8, 48, 64), t, w.num_samples, w.z_near, w.z_far, w.mu)
             for t in tg] for m in maps]
    for v in range(7):
        outs = [[(torch.empty((t.height, t.width), device="cuda"), torch.empty((t.height, t.width),
                 dtype=torch.int16, device="cuda")) for t in tg] for _ in maps]
        items = [(maps[f], t, outs[f][n][0], outs[f][n][1]) for f in range(2) for n, t in enumerate(tg)]
        b = gvs.FuseBatch(w.inputs, items, w.num_samples, w.z_near, w.z_far, w.mu, variant=v)
        b.launch()
        b.launch()  # the counter resets between launches
        torch.cuda.synchronize()
        for f in range(2):
            for n in range(len(tg)):
                assert torch.equal(outs[f][n][0].view(torch.int32), refs[f][n][0].view(torch.int32)), (v, f, n)
                assert torch.equal(outs[f][n][1], refs[f][n][1]), (v, f, n)
        b.close()


def test_batch_plan_graph_matches_single_view_api(gvs, tmp_path, monkeypatch):
    from paper_2505_18932_gb300 import autotune, batch
    from synth import configs
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "autotune.json"))
    w = configs.tiny(64, 48, 8, 96)
    tg = _targets(w)
    rgb0, d0 = w.render_inputs(0)
    frames = [w.render_inputs(f) for f in (1, 2)]
    rgba = [to_dev(u32(r)) for r, _ in frames]
    dep = [to_dev(d) for _, d in frames]
    plan = batch.BatchPlan(w.inputs, tg, rgba, dep, w.num_samples, w.z_near, w.z_far, w.mu, tau=w.tau,
                           rgba_prev=to_dev(u32(rgb0)), state0=to_dev(d0), variant=None, graph=True)
    assert plan.variant in range(7)
    cache = json.load(open(autotune.CACHE_PATH))
    assert any(e["variant"] == plan.variant for e in cache.values())
    for rep in range(2):
        plan.run()
    torch.cuda.synchronize()
    # the same frames through the single-view API, eagerly
    state = to_dev(d0)
    prev = to_dev(u32(rgb0))
    for f in range(2):
        gvs.refine_depth(rgba[f], prev, dep[f], state, tau=w.tau)
        prev = rgba[f]
        assert torch.equal(state, plan.states[f])
        for n, t in enumerate(tg):
            fu, cr = gvs.fuse_depth(w.inputs, state, t, w.num_samples, w.z_near, w.z_far, w.mu)
            sp = gvs.forward_splat(w.inputs, state, rgba[f], t, fused=fu, mu_guide=w.mu)
            torch.cuda.synchronize()
            assert torch.equal(fu.view(torch.int32), plan.fused[f][n].view(torch.int32))
            assert torch.equal(cr, plan.cross[f][n])
            for k in sp:
                assert torch.equal(sp[k], plan.splat[f][n][k]), (f, n, k)
