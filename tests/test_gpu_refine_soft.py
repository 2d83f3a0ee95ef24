"""The paper's soft difference mask on the GPU (gvs_refine_depth_soft) against the
FP64 oracle: mask within 1e-6 absolute, filtered depth within 1e-6 relative."""
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


@pytest.mark.parametrize("shape", [(2, 37, 53), (8, 720, 1280)])
def test_soft_refine_matches_oracle(gvs, oracle_mod, shape):
    N, H, W = shape
    rng = np.random.default_rng(H)
    a = rng.integers(0, 256, (N, H, W, 4), dtype=np.uint8)
    b = a.copy()
    sel = rng.random((N, H, W)) < 0.1
    b[sel] = rng.integers(0, 256, (int(sel.sum()), 4), dtype=np.uint8)
    d = rng.uniform(0.5, 6.0, (N, H, W)).astype(np.float32)
    p = rng.uniform(0.5, 6.0, (N, H, W)).astype(np.float32)
    d[rng.random((N, H, W)) < 0.01] = 0.0
    p[rng.random((N, H, W)) < 0.01] = np.nan
    ref, mref = oracle_mod.refine_depth_soft(b, a, d, p)
    st = to_dev(p)
    m = torch.empty((N, H, W), device="cuda")
    gvs.refine_depth_soft(to_dev(u32(b)), to_dev(u32(a)), to_dev(d), st, m)
    torch.cuda.synchronize()
    assert np.abs(m.cpu().numpy() - mref).max() <= 1e-6
    got = st.cpu().numpy().astype(np.float64)
    ok = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), ok)
    np.testing.assert_allclose(got[ok], ref[ok], rtol=1e-6)


def test_soft_refine_video_frames_f16(gvs, oracle_mod):
    from synth import configs
    w = configs.video_8x720p()
    rgb0, d0 = w.render_inputs(4)
    rgb1, d1 = w.render_inputs(5)
    d0h, d1h = d0.astype(np.float16), d1.astype(np.float16)
    ref, _ = oracle_mod.refine_depth_soft(rgb1, rgb0, d1h.astype(np.float32), d0h.astype(np.float32))
    st = torch.from_numpy(d0h.copy()).cuda()
    gvs.refine_depth_soft(to_dev(u32(rgb1)), to_dev(u32(rgb0)), torch.from_numpy(d1h).cuda(), st)
    torch.cuda.synchronize()
    got = st.cpu().numpy().astype(np.float64)
    # the FP16 state rounds the blended depth once: half an FP16 ulp relative
    np.testing.assert_allclose(got, ref, rtol=2.0 ** -11)
