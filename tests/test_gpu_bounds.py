"""The bounds-checked debug library (GVS_BOUNDS_CHECK): every entry point with
computed gather / scatter indices runs on real workloads, records no
out-of-range index, and gives the same results as the normal library."""
import numpy as np
import pytest
import torch

from gpu_util import to_dev, u32

pytestmark = pytest.mark.gpu


def _run_all(gvs, w):
    rgb, d = w.render_inputs(0)
    tgt = w.targets[0]
    dd, cc = to_dev(d), to_dev(u32(rgb))
    fused, cross = gvs.fuse_depth(w.inputs, dd, tgt, w.num_samples, w.z_near, w.z_far, w.mu)
    sp = gvs.forward_splat(w.inputs, dd, cc, tgt, fused=fused, mu_guide=w.mu)
    rej = gvs.forward_splat(w.inputs, dd, cc, tgt, fused=fused, mu_guide=w.mu, guide_reject=True)
    col, gdep = gvs.gauss_splat(w.inputs, dd, cc, tgt)
    sf, se = gvs.fuse_depth_sphere(w.inputs, dd, tgt, w.z_near, w.z_far, w.mu)
    dg = dd.clone().requires_grad_(True)
    f2, _ = gvs.FuseDepth.apply(dg, w.inputs, tgt, dict(num_samples=w.num_samples, z_near=w.z_near,
                                                         z_far=w.z_far, mu=w.mu))
    f2.sum().backward()
    torch.cuda.synchronize()
    return [fused, cross, sp["winner"], sp["warped_rgba"], sp["guided"], rej["winner"], col, gdep, sf, se, dg.grad]


@pytest.mark.parametrize("name", ["tiny", "plain_320x240"])
def test_checked_build_records_nothing_and_matches(name):
    from paper_2505_18932_gb300 import build as B, gvs
    from synth import configs
    w = configs.tiny(70, 45, 3, 96) if name == "tiny" else configs.plain_320x240()
    gvs._lib = None
    gvs.load()
    normal = _run_all(gvs, w)
    assert gvs.load().gvs_debug_bounds_error() == 0          # the normal build checks nothing
    checked_path = B.build(bounds_check=True)
    try:
        gvs._lib = None
        gvs.load(checked_path)
        lib = gvs.load()
        assert lib.gvs_debug_bounds_error() == 0
        checked = _run_all(gvs, w)
        err = lib.gvs_debug_bounds_error()
        assert err == 0, f"site {err >> 48}, index {err & ((1 << 48) - 1)}"
    finally:
        gvs._lib = None
        gvs.load()
    for i, (a, b) in enumerate(zip(normal, checked)):
        if i == len(normal) - 1:      # the fusion adjoint uses float atomics: equal up to their order
            torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6 * float(a.abs().max()))
        else:
            assert torch.equal(a, b), i
