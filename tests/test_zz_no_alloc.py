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


def _drv():
    """The CUDA driver library, for making a context of the test's own."""
    cu = ctypes.CDLL("libcuda.so.1")
    for name in ("cuInit", "cuDeviceGet", "cuCtxCreate_v2", "cuCtxDestroy_v2", "cuCtxSynchronize", "cuMemAlloc_v2",
                 "cuMemFree_v2", "cuMemcpyHtoD_v2", "cuMemcpyDtoH_v2"):
        getattr(cu, name).restype = ctypes.c_int
    return cu


def test_noalloc_in_a_context_the_caller_created():
    """A host application may run the library inside a context it created itself
    instead of the device's primary context.  Each context holds its own copy of
    the fixed z-buffer, so the call must use the copy of the context current at
    the call.  The library first runs in the primary context (caching that
    context's copy), then in a new context with every array allocated there, and
    then in the primary context again; all three agree bit for bit with the
    workspace splat."""
    from paper_2505_18932_gb300 import gvs
    lib = gvs.load()
    w, depth, rgba, fused = _inputs("plain_320x240")
    tgt = w.targets[0]
    ref = gvs.forward_splat(w.inputs, depth, rgba, tgt, fused=fused, mu_guide=w.mu)
    outs = {k: torch.full_like(v, 7) for k, v in ref.items()}
    _noalloc(lib, gvs, w, depth, rgba, fused, outs)   # primary context: caches its copy
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(outs[k], ref[k]), ("primary", k)
    host_in = {"depth": depth.cpu().numpy(), "rgba": rgba.cpu().numpy(), "fused": fused.cpu().numpy()}
    host_ref = {k: v.cpu().numpy() for k, v in ref.items()}

    cu = _drv()
    assert cu.cuInit(0) == 0
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    ctx = ctypes.c_void_p()
    assert cu.cuCtxCreate_v2(ctypes.byref(ctx), 0, dev) == 0   # current on this thread from here
    ptrs = {}
    try:
        def alloc(name, nbytes):
            p = ctypes.c_uint64()
            assert cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nbytes)) == 0
            ptrs[name] = p.value
            return p.value
        for k, a in host_in.items():
            a = np.ascontiguousarray(a)
            assert cu.cuMemcpyHtoD_v2(ctypes.c_uint64(alloc(k, a.nbytes)), a.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_size_t(a.nbytes)) == 0
        for k, a in host_ref.items():
            alloc("out_" + k, a.nbytes)
        p = gvs.GvsSplatParams(1, 2.0, float(w.mu))
        st = lib.gvs_forward_splat_noalloc(gvs.camera_array(w.inputs), ctypes.c_void_p(ptrs["depth"]),
                                           ctypes.c_void_p(ptrs["rgba"]), len(w.inputs),
                                           ctypes.byref(gvs.camera_struct(tgt)), ctypes.byref(p),
                                           ctypes.c_void_p(ptrs["fused"]), ctypes.c_void_p(ptrs["out_winner"]),
                                           ctypes.c_void_p(ptrs["out_warped_rgba"]),
                                           ctypes.c_void_p(ptrs["out_warped_depth"]),
                                           ctypes.c_void_p(ptrs["out_alpha"]), ctypes.c_void_p(ptrs["out_guided"]),
                                           None)
        assert st == 0, lib.gvs_last_error()
        assert cu.cuCtxSynchronize() == 0
        for k, a in host_ref.items():
            got = np.empty_like(a)
            assert cu.cuMemcpyDtoH_v2(got.ctypes.data_as(ctypes.c_void_p), ctypes.c_uint64(ptrs["out_" + k]),
                                      ctypes.c_size_t(a.nbytes)) == 0
            assert np.array_equal(got, a), ("own context", k)
    finally:
        for v in ptrs.values():
            cu.cuMemFree_v2(ctypes.c_uint64(v))
        assert cu.cuCtxDestroy_v2(ctx) == 0   # pops it: the primary context is current again

    outs = {k: torch.full_like(v, 7) for k, v in ref.items()}
    _noalloc(lib, gvs, w, depth, rgba, fused, outs)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(outs[k], ref[k]), ("primary again", k)
