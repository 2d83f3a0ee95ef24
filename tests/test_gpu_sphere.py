"""GPU parity of the sphere-tracing raymarch (Supplement A.1) against the
oracle: the march is FP32 on both sides with every operation rounded as
written and correctly rounded weights, so depths and evaluation counts are
compared bit for bit."""
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


def _case(gvs, oracle_mod, w, frame=0, half=False, **kw):
    _, d = w.render_inputs(frame)
    if half:
        d = d.astype(np.float16).astype(np.float32)
    tgt = w.targets_at(frame)[0]
    dd = to_dev(d).half() if half else to_dev(d)
    fused, evals = gvs.fuse_depth_sphere(w.inputs, dd, tgt, w.z_near, w.z_far, w.mu, **kw)
    torch.cuda.synchronize()
    ref = oracle_mod.fuse_depth_sphere(w.inputs, d, tgt, w.z_near, w.z_far, w.mu, **kw)
    g = fused.cpu().numpy()
    bad = g.view(np.uint32) != ref["depth"].view(np.uint32)
    assert not bad.any(), f"{bad.sum()} px differ, e.g. {np.argwhere(bad)[:3].tolist()}"
    assert np.array_equal(evals.cpu().numpy(), ref["evals"])
    return ref


def test_sphere_tiny_ragged(gvs, oracle_mod):
    from synth import configs
    ref = _case(gvs, oracle_mod, configs.tiny(70, 45, 3, 24))
    assert (ref["depth"] > 0).mean() > 0.5


def test_sphere_plain_320x240(gvs, oracle_mod):
    from synth import configs
    _case(gvs, oracle_mod, configs.plain_320x240())


@pytest.mark.parametrize("K", [1, 5, 12])
def test_sphere_view_counts(gvs, oracle_mod, K):
    from synth import configs
    _case(gvs, oracle_mod, configs.tiny(48, 40, K, 16))


def test_sphere_step_cap_and_min_step(gvs, oracle_mod):
    from synth import configs
    _case(gvs, oracle_mod, configs.tiny(64, 48, 3, 16), max_steps=20, min_frac=0.25)


def test_sphere_f16_depth(gvs, oracle_mod):
    from synth import configs
    _case(gvs, oracle_mod, configs.tiny(70, 45, 3, 24), half=True)


def test_sphere_video_720p_full(gvs, oracle_mod):
    """8 x 1280x720 inputs: every ray of the target compared bit for bit."""
    from synth import configs
    _case(gvs, oracle_mod, configs.video_8x720p(), frame=3)
