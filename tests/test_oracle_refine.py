"""Pins for the oracle's temporal depth refinement (Sec. 3.2, Eq. 1-2, binary form)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "refine_binary.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        a = lhs.split()
        b = rhs.split()
        rows.append((float(a[0]), [int(x) for x in a[1:5]], [int(x) for x in a[5:9]], float(a[9]), float(a[10]),
                     int(b[0]), float(b[1])))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_refine_hand_worked(oracle_mod, row):
    tau, rt, rp, dt, sp, m_exp, s_exp = row
    rgba_t = np.array(rt, np.uint8).reshape(1, 1, 1, 4)
    rgba_p = np.array(rp, np.uint8).reshape(1, 1, 1, 4)
    out, mask = oracle_mod.refine_depth(rgba_t, rgba_p, np.full((1, 1, 1), dt, np.float32),
                                        np.full((1, 1, 1), sp, np.float32), tau)
    assert int(mask[0, 0, 0]) == m_exp
    assert out[0, 0, 0] == np.float32(s_exp)


def test_first_frame_takes_new_depth(oracle_mod, synth_mod):
    from synth import configs
    w = configs.tiny(40, 24, 2)
    rgb, d = w.render_inputs(0)
    out, mask = oracle_mod.refine_depth(rgb, None, d, None, 0.03)
    assert mask.min() == 1
    assert np.array_equal(out.view(np.uint32), d.view(np.uint32))


def test_moving_sphere_static_background_unchanged(oracle_mod, synth_mod):
    """Only a sphere moves: wherever neither frame shows the sphere the colour is
    unchanged, so the mask is 0 and the previous depth is kept bit for bit; where
    the sphere covers one frame but not the other the colour changes and the
    mask must fire wherever that change exceeds the threshold."""
    from synth import Scene, render
    from synth import configs
    w = configs.video_8x720p()
    cam = w.inputs[0].__class__(**{**w.inputs[0].__dict__})
    cam.width, cam.height = 160, 90
    cam.fx, cam.fy, cam.cx, cam.cy = cam.fx / 8, cam.fy / 8, (160 - 1) / 2, (90 - 1) / 2
    sc0, sc1 = w.scene(3), w.scene(4)
    rgb0, d0 = render(sc0, cam, noise_seed=1, noise_sigma=0.002)
    rgb1, d1 = render(sc1, cam, noise_seed=2, noise_sigma=0.002)
    # sphere coverage from noise-free renders with and without the sphere
    bg = Scene(planes=sc0.planes, spheres=[], tex_seed=sc0.tex_seed)
    _, dbg = render(bg, cam)
    _, c0 = render(sc0, cam)
    _, c1 = render(sc1, cam)
    sphere_any = (c0 != dbg) | (c1 != dbg)
    assert sphere_any.any() and (~sphere_any).any()
    prev_state = d0.copy()
    out, mask = oracle_mod.refine_depth(rgb1[None], rgb0[None], d1[None], prev_state[None], 0.03)
    out, mask = out[0], mask[0]
    assert mask[~sphere_any].max() == 0
    assert np.array_equal(out[~sphere_any].view(np.uint32), prev_state[~sphere_any].view(np.uint32))
    big = np.abs(rgb1[..., :3].astype(int) - rgb0[..., :3].astype(int)).max(-1) > 7
    assert big.any()
    assert mask[big].min() == 1
    assert np.array_equal(out[big].view(np.uint32), d1[big].view(np.uint32))
