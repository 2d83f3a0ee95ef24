"""Host-side shape checks of the Python binding.  The C ABI takes every image
size from the cameras (or from explicit sizes), never from the arrays, so an
array of the wrong shape would be read or written past its end; the binding
refuses such calls with ValueError before anything reaches the library's
compute entry points.  The tensors here live on the CPU: every call must fail
on its shape check, before any device pointer is taken."""
import pytest
import torch


@pytest.fixture(scope="module")
def gvs():
    from paper_2505_18932_gb300 import build as b
    b.build()
    from paper_2505_18932_gb300 import gvs as g
    g.load()
    return g


@pytest.fixture(scope="module")
def scene():
    from synth import camera_at
    cams = [camera_at(40, 24, (0.1 * k, 0.0, 0.0)) for k in range(3)]
    tgt = camera_at(32, 20, (0.05, 0.0, -1.0))
    return cams, tgt


def _z(*shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype)


def test_soft_splat_colour_must_have_four_channels(gvs, scene):
    cams, tgt = scene
    d = _z(3, 24, 40)
    for bad in (_z(3, 24, 40), _z(3, 24, 40, 3), _z(3, 24, 40, dtype=torch.bfloat16)):
        with pytest.raises(ValueError, match="in_color"):
            gvs.soft_splat(cams, d, bad, tgt)
        with pytest.raises(ValueError, match="in_color"):
            gvs.soft_splat_backward(cams, d, bad, tgt, {}, _z(3, 20, 32, 4))


def test_depth_shape_follows_the_cameras(gvs, scene):
    cams, tgt = scene
    for bad in (_z(2, 24, 40), _z(3, 40, 24), _z(3, 24, 41)):
        with pytest.raises(ValueError, match="in_depths"):
            gvs.soft_splat(cams, bad, _z(*bad.shape, 4), tgt)
        with pytest.raises(ValueError, match="in_depths"):
            gvs.forward_splat(cams, bad, _z(*bad.shape, dtype=torch.int32), tgt)
        with pytest.raises(ValueError, match="in_depths"):
            gvs.fuse_depth(cams, bad, tgt, 64, 0.5, 5.0, 0.05)
        with pytest.raises(ValueError, match="in_depths"):
            gvs.fuse_depth_sphere(cams, bad, tgt, 0.5, 5.0, 0.05)
        with pytest.raises(ValueError, match="in_depths"):
            gvs.gauss_splat(cams, bad, _z(*bad.shape, dtype=torch.int32), tgt)


def test_rgba_bytes_per_pixel(gvs, scene):
    cams, tgt = scene
    d = _z(3, 24, 40)
    # packed int32 and uint8 [..., 4] hold the same bytes; a single uint8 plane does not
    with pytest.raises(ValueError, match="in_rgba"):
        gvs.forward_splat(cams, d, _z(3, 24, 40, dtype=torch.uint8), tgt)
    with pytest.raises(ValueError, match="in_rgba"):
        gvs.gauss_splat(cams, d, _z(3, 24, 40, 3, dtype=torch.uint8), tgt)
    with pytest.raises(ValueError, match="rgba_prev"):
        gvs.refine_depth(_z(3, 24, 40, dtype=torch.int32), _z(3, 24, 20, dtype=torch.int32), d, d.clone())


def test_caller_outputs_checked(gvs, scene):
    cams, tgt = scene
    d = _z(3, 24, 40)
    rgba = _z(3, 24, 40, dtype=torch.int32)
    with pytest.raises(ValueError, match="winner"):
        gvs.forward_splat(cams, d, rgba, tgt, outputs={"winner": _z(3, 20, 31, dtype=torch.int32)})
    with pytest.raises(ValueError, match="fused"):
        gvs.forward_splat(cams, d, rgba, tgt, fused=_z(20, 31))
    with pytest.raises(ValueError, match="color"):
        gvs.soft_splat(cams, d, _z(3, 24, 40, 4), tgt, outputs={"color": _z(3, 20, 32)})
    with pytest.raises(ValueError, match="fused"):
        gvs.fuse_depth(cams, d, tgt, 64, 0.5, 5.0, 0.05, fused=_z(32, 20))
    with pytest.raises(ValueError, match="crossing"):
        gvs.fuse_depth(cams, d, tgt, 64, 0.5, 5.0, 0.05, crossing=_z(20, 32))
    with pytest.raises(ValueError, match="shape"):
        gvs.fuse_depth_from_map(cams, _z(1024, dtype=torch.uint8), (3, 24, 41), tgt, 64, 0.5, 5.0, 0.05)
    with pytest.raises(ValueError, match="mask"):
        gvs.refine_depth(rgba, rgba, d, d.clone(), mask=_z(3, 24, 40))


def test_blend_planes_checked(gvs):
    K, Ht, Wt = 2, 20, 32
    rgba = _z(K, Ht, Wt, dtype=torch.int32)
    a = _z(K, Ht, Wt, dtype=torch.uint8)
    wd = _z(K, Ht, Wt)
    with pytest.raises(ValueError, match="i_bg"):
        gvs.blend(rgba, a, wd, _z(Ht, Wt), _z(K, Ht, Wt), _z(Ht, Wt), _z(Ht, Wt))
    with pytest.raises(ValueError, match="fused"):
        gvs.blend(rgba, a, wd, _z(Ht, Wt + 1), _z(K, Ht, Wt), _z(Ht, Wt), _z(3, Ht, Wt))
    with pytest.raises(ValueError, match="alpha"):
        gvs.guided_mask(wd, _z(K, Ht, Wt + 1, dtype=torch.uint8), _z(Ht, Wt), 0.05)


def test_valid_shapes_pass_the_checks(gvs, scene):
    """Correctly shaped CPU tensors get past every shape check and stop only at the
    device check (optional arguments left out, as the header allows)."""
    cams, tgt = scene
    d = _z(3, 24, 40)
    rgba = _z(3, 24, 40, dtype=torch.int32)
    rgba8 = _z(3, 24, 40, 4, dtype=torch.uint8)
    calls = [
        lambda: gvs.refine_depth(rgba, None, d, d.clone()),
        lambda: gvs.refine_depth(rgba8, rgba, d, d.clone(), mask=_z(3, 24, 40, dtype=torch.uint8)),
        lambda: gvs.forward_splat(cams, d, rgba8, tgt, fused=_z(20, 32)),
        lambda: gvs.soft_splat(cams, d, _z(3, 24, 40, 4, dtype=torch.bfloat16), tgt),
        lambda: gvs.fuse_depth(cams, d.half(), tgt, 64, 0.5, 5.0, 0.05),
        lambda: gvs.fuse_depth_sphere(cams, d, tgt, 0.5, 5.0, 0.05),
        lambda: gvs.gauss_splat(cams, d, rgba, tgt),
        lambda: gvs.blend(_z(3, 20, 32, dtype=torch.int32), _z(3, 20, 32, dtype=torch.uint8), _z(3, 20, 32),
                          _z(20, 32), _z(3, 20, 32), _z(20, 32), _z(3, 20, 32)),
        lambda: gvs.guided_mask(_z(3, 20, 32), _z(3, 20, 32, dtype=torch.uint8), _z(20, 32), 0.05),
    ]
    for c in calls:
        with pytest.raises(ValueError, match="CUDA device"):
            c()
