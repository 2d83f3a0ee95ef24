"""gvs_forward_splat_noalloc: the splat for callers that cannot allocate device memory.

A plugin inside a host application that owns every device allocation, code
recorded into a CUDA graph, or a real-time loop that must not block on the
allocator cannot create the splat workspace.  This entry point keeps its
z-buffer in a fixed device array inside the library instead.  The test calls
it through the C ABI twice in a row (the array keeps the previous call's
contents, so the second call checks that it is cleared) and compares every
output with gvs_forward_splat on a caller-provided workspace; the splat
outputs are integer maps and copies, so they must agree bit for bit.

This file is collected last so that a failure here stops a `-x` run only
after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(name):
    from synth import configs
    w = getattr(configs, name)()
    rgb, d = w.render_inputs(1)
    tgt = w.targets[0]
    _, gt = w.render_target_gt(tgt, 1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return (w, dev(d), dev(np.ascontiguousarray(rgb).view(np.int32)[..., 0]), dev(gt.astype(np.float32)))


def _noalloc(lib, gvs, w, depth, rgba, fused, outs):
    p = gvs.GvsSplatParams(1, 2.0, float(w.mu))
    tgt = w.targets[0]
    st = lib.gvs_forward_splat_noalloc(gvs.camera_array(w.inputs), depth.data_ptr(), rgba.data_ptr(),
                                       len(w.inputs), ctypes.byref(gvs.camera_struct(tgt)), ctypes.byref(p),
                                       fused.data_ptr(), outs["winner"].data_ptr(), outs["warped_rgba"].data_ptr(),
                                       outs["warped_depth"].data_ptr(), outs["alpha"].data_ptr(),
                                       outs["guided"].data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.gvs_last_error()


@pytest.mark.parametrize("name", ["plain_320x240", "headline_8x1080p"])
def test_noalloc_matches_workspace_splat_twice(name):
    from paper_2505_18932_gb300 import gvs
    lib = gvs.load()
    w, depth, rgba, fused = _inputs(name)
    ref = gvs.forward_splat(w.inputs, depth, rgba, w.targets[0], fused=fused, mu_guide=w.mu)
    for call in range(2):
        outs = {k: torch.full_like(v, 7) for k, v in ref.items()}
        _noalloc(lib, gvs, w, depth, rgba, fused, outs)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(outs[k], ref[k]), (name, call, k)


def test_noalloc_rejects_targets_beyond_its_buffer():
    from paper_2505_18932_gb300 import gvs
    from synth import camera_at
    lib = gvs.load()
    big = camera_at(2049, 1024, (0.0, 0.0, 0.0))   # 2,098,176 pixels > 2^21
    p = gvs.GvsSplatParams(1, 2.0, 0.04)
    st = lib.gvs_forward_splat_noalloc(gvs.camera_array([big]), 0x10000, 0x10000, 1, ctypes.byref(gvs.camera_struct(big)),
                                       ctypes.byref(p), None, 0x10000, None, None, None, None, None)
    assert st == 1
    assert b"at most" in lib.gvs_last_error()
