"""The differentiable workload's own loss, checked by central finite differences.

4 input views at 640x360 (the arc rig), one target between them, the
differentiable colour splat of every view, blended with uniform weights
(Eq. 4 with w_k = 1: B = sum_k alpha_k I_k / sum_k alpha_k) and compared with
the ground-truth render of the target: L = mean over covered pixels and the
three channels of |B - GT|.  The oracle's adjoint (soft_splat_grad fed with
dL/dI_k = alpha_k / sum alpha * sign(B - GT) / (3 n)) must agree with
(L(x + h) - L(x - h)) / 2h at 64 seeded input pixels, h = 1e-3 m on depth and
h = 1e-3 on colour, within 1e-2 of the larger magnitude.

Only the differentiated view is re-splatted for each difference.  A pixel
whose difference changes between h and h / 2 (a footprint bound, the front
band, a winner or an L1 sign flipping inside the step) sits on a kink and is
redrawn from the next seed, and so is one where some blended value B - GT
changes sign (or is 0) within the step, the kink of |B - GT|; the count of
redraws is bounded.  Depth pixels
are drawn among those the target sees (a non-zero adjoint), so that every
check is informative.
"""
import numpy as np
import pytest

H_DEPTH = 1e-3
H_COLOR = 1e-3
N_PIXELS = 64


@pytest.fixture(scope="module")
def case(oracle_mod, synth_mod):
    from synth import configs
    w = configs.diff_640x360()
    rgb, d = w.render_inputs(0)
    tgt = w.targets[0]
    gt_rgb, _ = w.render_target_gt(tgt, 0)
    gt = np.asarray(gt_rgb[..., :3], np.float64) / 255.0
    col = np.asarray(rgb, np.float64) / 255.0
    return w, tgt, d.copy(), col, gt


def _splat(oracle_mod, w, tgt, d, col, views):
    cams = [w.inputs[k] for k in views]
    s = oracle_mod.soft_splat(cams, np.ascontiguousarray(d[views]), np.ascontiguousarray(col[views]), tgt,
                              mu_band=w.mu)
    return s["color"][..., :3], s["alpha"].astype(np.float64)


def _blend(I, A):
    asum = A.sum(0)
    return (I * A[..., None]).sum(0) / np.maximum(asum, 1.0)[..., None], asum > 0


def _loss(I, A, gt):
    B, cov = _blend(I, A)
    return np.abs(B - gt)[cov].sum() / (3.0 * cov.sum())


def _adjoint(oracle_mod, w, tgt, d, col, gt):
    N = len(w.inputs)
    I, A = _splat(oracle_mod, w, tgt, d, col, list(range(N)))
    asum = A.sum(0)
    cov = asum > 0
    B = (I * A[..., None]).sum(0) / np.maximum(asum, 1.0)[..., None]
    up = np.sign(B - gt) * cov[..., None] / (3.0 * cov.sum())
    gcol = np.zeros(I.shape[:-1] + (4,))
    gcol[..., :3] = (A / np.maximum(asum, 1.0))[..., None] * up[None]
    gd, gc = oracle_mod.soft_splat_grad(w.inputs, d, col, tgt, gcol, None, mu_band=w.mu)
    return I, A, gd, gc


def _differences(oracle_mod, w, tgt, d, col, gt, I, A, k, field, idx, h):
    """Central difference of L for one input value (view k re-splatted), and whether some
    blended value B - GT changes sign (or is 0) within the step: the kink of |B - GT|."""
    vals, dev = [], []
    for sgn in (1.0, -1.0):
        dd, cc = d.copy(), col.copy()
        if field == "depth":
            dd[(k,) + idx] = np.float32(d[(k,) + idx] + sgn * h)
        else:
            cc[(k,) + idx] += sgn * h
        Ik, Ak = _splat(oracle_mod, w, tgt, dd, cc, [k])
        I2, A2 = I.copy(), A.copy()
        I2[k], A2[k] = Ik[0], Ak[0]
        vals.append(_loss(I2, A2, gt))
        B, cov = _blend(I2, A2)
        dev.append(np.where(cov[..., None], B - gt, 1.0))
    if field == "depth":  # the steps actually taken in FP32 storage
        hp = float(np.float32(d[(k,) + idx] + h)) - float(d[(k,) + idx])
        hm = float(d[(k,) + idx]) - float(np.float32(d[(k,) + idx] - h))
    else:
        hp = hm = h
    B0, cov0 = _blend(I, A)
    d0 = np.where(cov0[..., None], B0 - gt, 1.0)
    moved = (dev[0] != d0) | (dev[1] != d0)
    flip = bool(((dev[0] * dev[1] <= 0.0) & moved).any() or ((d0 == 0.0) & moved).any())
    return (vals[0] - vals[1]) / (hp + hm), flip


def _check(oracle_mod, case, field):
    w, tgt, d, col, gt = case
    I, A, gd, gc = _adjoint(oracle_mod, w, tgt, d, col, gt)
    N, Hs, Ws = d.shape
    if field == "depth":
        g = gd
        cand = np.argwhere(np.abs(gd) > 1e-3 * np.abs(gd).max())
        h = H_DEPTH
    else:
        g = gc[..., :3]
        cand = np.argwhere(np.abs(g) > 1e-3 * np.abs(g).max())
        h = H_COLOR
    rng = np.random.default_rng(2025)
    done, redrawn = 0, 0
    while done < N_PIXELS:
        assert redrawn <= N_PIXELS, f"{redrawn} kinked draws for {done} clean ones"
        pick = tuple(cand[rng.integers(len(cand))])
        k, idx = int(pick[0]), tuple(int(x) for x in pick[1:])
        fd, flip = _differences(oracle_mod, w, tgt, d, col, gt, I, A, k, field, idx, h)
        fd2, _ = _differences(oracle_mod, w, tgt, d, col, gt, I, A, k, field, idx, h / 2)
        # a kink inside the step: an L1 sign flips, or the halved step disagrees (a footprint
        # bound, the front band or a winner changed)
        if flip or abs(fd - fd2) > 1e-2 * max(abs(fd), abs(fd2), 1e-30):
            redrawn += 1
            continue
        ref = g[(k,) + idx]
        assert abs(fd2 - ref) <= 1e-2 * max(abs(ref), abs(fd2)), (field, k, idx, fd2, ref)
        done += 1
    print(f"{field}: {done} pixels checked, {redrawn} redrawn on kinks")
    return redrawn


def test_depth_gradient_matches_central_differences(oracle_mod, case):
    _check(oracle_mod, case, "depth")


def test_colour_gradient_matches_central_differences(oracle_mod, case):
    _check(oracle_mod, case, "color")
