"""Helpers shared by the GPU parity tests: seeded inputs on the device and
the comparison rules (bit-exact integer maps; 1e-4 relative fused depth on
pixels the oracle does not flag as ambiguous)."""
import numpy as np
import torch

import os

DEPTH_RTOL = 1e-4          # fused depth, FP32 kernel vs FP64 oracle
MAX_AMBIGUOUS = 1e-3       # flagged-pixel fraction above which a case fails

# (test id, flagged pixels, compared pixels) of every fused-depth comparison in
# this session; the terminal summary of the run reports them
AMBIGUOUS_LOG = []


def u32(rgba):
    """[..., 4] uint8 -> [...] uint32 packed RGBA8."""
    return np.ascontiguousarray(rgba).view(np.uint32)[..., 0]


def to_dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def compare_fused(gpu_depth, gpu_index, ref, where=None):
    """Assert fused-depth parity; returns the ambiguous fraction."""
    gd = gpu_depth.cpu().numpy().astype(np.float64)
    gi = gpu_index.cpu().numpy().astype(np.int32) if gpu_index is not None else None
    rd, ri, amb = ref["depth"], ref["index"], ref["ambiguous"].astype(bool)
    if where is not None:
        gd = gd[where]
        gi = gi[where] if gi is not None else None
    ok = ~amb
    if gi is not None:
        bad = ok & (gi != ri)
        assert not bad.any(), f"crossing index differs at {np.argwhere(bad)[:5].tolist()} ({bad.sum()} px)"
    err = np.abs(gd - rd)
    tol = DEPTH_RTOL * np.abs(rd)
    bad = ok & (err > tol)
    assert not bad.any(), (f"fused depth differs at {bad.sum()} px, worst rel "
                           f"{(err[bad] / np.maximum(np.abs(rd[bad]), 1e-30)).max():.3e}")
    frac = amb.mean() if amb.size else 0.0
    AMBIGUOUS_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], int(amb.sum()), int(amb.size)))
    assert frac <= MAX_AMBIGUOUS, f"ambiguous fraction {frac:.2e} ({int(amb.sum())} of {amb.size} px)"
    return frac
