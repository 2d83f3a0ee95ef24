"""The temporal term (Sec. 3.2, Supplement A.2) on the GPU against the FP64 oracle:
the weight (1e-6), fusion with the previous output as an input (same bar as the
plain fusion), the plane closed form, and a three-frame online sequence."""
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


@pytest.mark.parametrize("u8", [False, True])
def test_temporal_weight_matches_oracle(gvs, oracle_mod, u8):
    rng = np.random.default_rng(1 + u8)
    N, H, W, Ht, Wt = 3, 20, 30, 17, 23
    masks = (rng.random((N, H, W)) < 0.3).astype(np.uint8) if u8 else rng.uniform(0.6, 1.0, (N, H, W)).astype(np.float32)
    winner = rng.integers(-1, H * W, (N, Ht, Wt)).astype(np.int32)
    wp = rng.uniform(0, 10, (Ht, Wt)).astype(np.float32)
    wv = rng.uniform(0, 8, (Ht, Wt)).astype(np.float32)
    ref, M = oracle_mod.temporal_weight(masks.astype(np.float32), winner, wp, wv, 1.3, 15.0)
    tm = torch.empty((Ht, Wt), device="cuda")
    got = gvs.temporal_weight(to_dev(masks), to_dev(winner), to_dev(wp), to_dev(wv), 1.3, 15.0, target_mask=tm)
    torch.cuda.synchronize()
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(tm.cpu().numpy(), M, rtol=1e-7)


@pytest.mark.parametrize("shape", [(3, 20, 32), (4, 17, 23)])
def test_guided_mask_matches_definition(gvs, shape):
    """gvs_guided_mask (Sec. 3.3: the views' pixels within mu of the fused depth) bit for bit
    against the definition in FP64, on depths in [1, 2] where |d - F| is exact in FP32, with
    exact ties at mu planted; a target size divisible by 4 (four pixels per thread) and one
    that is not (one per thread)."""
    K, Ht, Wt = shape
    rng = np.random.default_rng(K * Ht)
    mu = 0.0625
    fused = rng.uniform(1.0, 2.0, (Ht, Wt)).astype(np.float32)
    wd = (fused[None] + rng.uniform(-0.2, 0.2, (K, Ht, Wt))).astype(np.float32)
    wd = np.clip(wd, 1.0, 2.0).astype(np.float32)
    tie = rng.random((K, Ht, Wt)) < 0.05
    wd[tie] = np.clip(fused[None].repeat(K, 0)[tie] + mu, 1.0, 2.0)
    alpha = (rng.random((K, Ht, Wt)) < 0.8).astype(np.uint8)
    g = gvs.guided_mask(to_dev(wd), to_dev(alpha), to_dev(fused), mu)
    torch.cuda.synchronize()
    ref = (alpha > 0) & (np.abs(wd.astype(np.float64) - fused.astype(np.float64)[None]) <= mu)
    assert np.array_equal(g.cpu().numpy(), ref.astype(np.uint8))
    assert ref.any() and (~ref & (alpha > 0)).any()


def test_fuse_temporal_matches_oracle(gvs, oracle_mod):
    from synth import configs
    w = configs.tiny(70, 45, 4, 96)
    _, d = w.render_inputs(0)
    t = w.targets[0]
    rng = np.random.default_rng(4)
    base = oracle_mod.fuse_depth(w.inputs, d, t, w.num_samples, w.z_near, w.z_far, w.mu)
    prev = (base["depth"] + rng.normal(0, 0.01, base["depth"].shape)).astype(np.float32)
    prev[base["index"] < 0] = 0.0
    wt = rng.uniform(0, 15, prev.shape).astype(np.float32)
    wt[rng.random(prev.shape) < 0.2] = 0.0
    ref = oracle_mod.fuse_depth_temporal(w.inputs, d, t, w.num_samples, w.z_near, w.z_far, w.mu, prev, wt)
    m = gvs.weight_map(to_dev(d), w.mu)
    f, c, wv = gvs.fuse_depth_temporal(w.inputs, m, t, w.num_samples, w.z_near, w.z_far, w.mu, to_dev(prev),
                                       to_dev(wt))
    torch.cuda.synchronize()
    compare_fused(f, c, ref)
    ok = (ref["ambiguous"] == 0) & (ref["index"] >= 0)
    np.testing.assert_allclose(wv.cpu().numpy()[ok], ref["wview"][ok], rtol=1e-4, atol=1e-5)


def test_fuse_temporal_plane_weighted_mean(gvs):
    from synth import camera_at
    cams = [camera_at(48, 32, (x, y, 0.0)) for x, y in [(-0.05, 0.0), (0.05, 0.0), (0.0, 0.04)]]
    tgt = camera_at(48, 32, (0.0, 0.0, 0.0))
    d1, d2, wt = 2.5, 2.52, 4.0
    m = gvs.weight_map(torch.full((3, 32, 48), d1, device="cuda"), 0.05)
    f, c, wv = gvs.fuse_depth_temporal(cams, m, tgt, 1024, 0.5, 5.0, 0.05, torch.full((32, 48), d2, device="cuda"),
                                       torch.full((32, 48), wt, device="cuda"))
    torch.cuda.synchronize()
    exp = (3 * float(np.float32(d1)) + wt * float(np.float32(d2))) / (3 + wt)
    np.testing.assert_allclose(f.cpu().numpy()[6:-6, 8:-8], exp, rtol=1e-5)
    np.testing.assert_allclose(wv.cpu().numpy()[6:-6, 8:-8], 3.0, rtol=1e-5)


def test_online_sequence_matches_oracle(gvs, oracle_mod):
    """Three frames of a moving sphere seen from a fixed novel viewpoint: binary
    difference masks (bit-exact refined depths on both sides), temporal weights and
    temporally fused depths against the oracle frame by frame (each frame's oracle
    inputs are its own previous outputs, never the GPU's)."""
    from synth import configs
    w = configs.tiny(64, 48, 4, 96)
    tgt = w.targets[0]
    frames = [w.render_inputs(f) for f in range(4)]
    tf = gvs.TemporalFusion(w.inputs, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    state_g = to_dev(frames[0][1])
    o_state = frames[0][1]
    o_prev = np.zeros((tgt.height, tgt.width), np.float32)
    o_wtmp = np.zeros_like(o_prev)
    o_wview = np.zeros_like(o_prev)
    for f in range(1, 4):
        rgb_p, rgb_c = frames[f - 1][0], frames[f][0]
        mask_g = torch.empty(state_g.shape, dtype=torch.uint8, device="cuda")
        gvs.refine_depth(to_dev(u32(rgb_c)), to_dev(u32(rgb_p)), to_dev(frames[f][1]), state_g, mask_g, tau=w.tau)
        fused, cross, sp, w_tmp = tf.step(state_g, to_dev(u32(rgb_c)), mask_g)
        torch.cuda.synchronize()
        o_state, o_mask = oracle_mod.refine_depth(rgb_c, rgb_p, frames[f][1], o_state, w.tau)
        hs = oracle_mod.forward_splat(w.inputs, o_state, u32(rgb_c), tgt)
        assert np.array_equal(sp["winner"].cpu().numpy(), hs["winner"])
        o_w, _ = oracle_mod.temporal_weight(o_mask.astype(np.float32), hs["winner"], o_wtmp, o_wview)
        ref = oracle_mod.fuse_depth_temporal(w.inputs, o_state, tgt, w.num_samples, w.z_near, w.z_far, w.mu, o_prev,
                                             o_w.astype(np.float32))
        np.testing.assert_allclose(w_tmp.cpu().numpy(), o_w, rtol=1e-5, atol=1e-4)
        compare_fused(fused, cross, ref)
        o_prev = ref["depth"].astype(np.float32)
        o_wtmp = o_w.astype(np.float32)
        o_wview = ref["wview"].astype(np.float32)


def test_checkpoint_resume_is_bit_identical(gvs):
    """Stop after frame 3, save the online state (the refined input depths and the
    temporal state) to the host, rebuild everything from it and continue: frames 4-6
    equal an uninterrupted run bit for bit."""
    from synth import configs
    w = configs.tiny(64, 48, 4, 96)
    tgt = w.targets[0]
    frames = [w.render_inputs(f) for f in range(7)]

    def run(f0, f1, state, tf):
        outs = []
        for f in range(f0, f1):
            rgb_p, rgb_c = frames[f - 1][0], frames[f][0]
            mask = torch.empty(state.shape, dtype=torch.uint8, device="cuda")
            gvs.refine_depth(to_dev(u32(rgb_c)), to_dev(u32(rgb_p)), to_dev(frames[f][1]), state, mask, tau=w.tau)
            fused, cross, sp, w_tmp = tf.step(state, to_dev(u32(rgb_c)), mask)
            outs.append([fused.clone(), cross.clone(), w_tmp.clone(), sp["guided"].clone()])
        return outs

    state = to_dev(frames[0][1])
    tf = gvs.TemporalFusion(w.inputs, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    full = run(1, 7, state, tf)
    state = to_dev(frames[0][1])
    tf = gvs.TemporalFusion(w.inputs, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    run(1, 4, state, tf)
    ckpt = {"refined": state.cpu(), "temporal": tf.state_dict()}
    del state, tf
    state = ckpt["refined"].cuda()
    tf = gvs.TemporalFusion(w.inputs, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    tf.load_state_dict(ckpt["temporal"])
    resumed = run(4, 7, state, tf)
    torch.cuda.synchronize()
    for a, b in zip(full[3:], resumed):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    assert (full[-1][2] > 0).any()     # the temporal term is active by then
