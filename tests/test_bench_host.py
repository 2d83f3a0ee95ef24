"""Host-side pieces of bench.py that its JSON line rests on: the algorithmic work
count behind `roofline`, the compulsory-byte accounting behind `hbm`, and the rule
that the committed ncu counter record is reported only for the kernel it was taken
from (same sources, same bundle shape).  No GPU."""
import importlib.util
import json
import os
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_fuse_counts_samples_up_to_the_second_bracket(bench):
    # crossing index s: samples 0..s+1 are needed (min with D); no crossing (-1): all D; times K views
    s = np.array([[0, -1], [5, 126]], np.int16)
    assert bench.algorithmic_fuse(s, 128, 8) == (2 + 128 + 7 + 128) * 8


def test_compulsory_bytes_per_stage(bench):
    N, H, W, Ht, Wt = 2, 3, 4, 5, 6
    px, tpx = N * H * W, Ht * Wt
    ab = bench.alg_bytes(N, H, W, Ht, Wt)
    # refine: two RGBA8 frames, depth and state in, state and mask out
    assert ab["refine"] == px * 16 + px * 5
    # weight map: depth in, (d, omega) float2 out
    assert ab["weight_map"] == px * 4 + px * 8
    # fusion: the map once, fused depth (f32) and crossing (i16) out
    assert ab["fuse"] == px * 8 + tpx * 6
    # splat: depth and colour in, per view and target pixel 14 bytes out, fused depth read once
    assert ab["splat"] == px * 8 + tpx * N * 14 + tpx * 4


def test_counter_record_only_for_its_own_kernel(bench, tmp_path, monkeypatch):
    """A record applies to the sources it names, hashed, and to one bundle shape; a stale
    record (bench then reports traffic as null) is no test failure."""
    import hashlib
    rec = json.load(open(os.path.join(ROOT, "profiles", "fuse_kernel_traffic.txt")))
    os.makedirs(tmp_path / "profiles")
    h = hashlib.sha256()
    for src in rec["source_files"]:
        dst = tmp_path / src
        os.makedirs(dst.parent, exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), dst)
        h.update(open(dst, "rb").read())
    rec.update({"source_sha256": h.hexdigest(), "variant": 3})
    with open(tmp_path / "profiles" / "fuse_kernel_traffic.txt", "w") as f:
        json.dump(rec, f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.recorded_counters(3)
    assert got is not None and got["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"]
    assert bench.recorded_counters(0) is None  # another bundle shape
    with open(tmp_path / rec["source_files"][0], "ab") as f:
        f.write(b"\n")
    assert bench.recorded_counters(3) is None  # the kernel's sources changed


def test_autotuner_chooses_only_between_distinct_kernels():
    """Bundle shapes are compiled for 5..16 views and the warp-per-ray mapping (variant 6)
    for 5..32; elsewhere every variant is the default kernel, so there is nothing to time
    and the default comes back at once."""
    from paper_2505_18932_gb300 import autotune
    assert autotune.variants_for(8) == autotune.VARIANTS and autotune.variants_for(16) == autotune.VARIANTS
    assert autotune.variants_for(5) == autotune.VARIANTS and 6 in autotune.VARIANTS
    for k in (17, 32):
        assert autotune.variants_for(k) == (0, 6)
    for k in (1, 4):
        assert autotune.variants_for(k) == (0,)
    calls = []
    best, ms = autotune.choose({"k": 4}, lambda v: calls.append(v), candidates=autotune.variants_for(4))
    assert best == 0 and ms == {} and calls == []


def test_roofline_fraction_is_an_issue_fraction(bench):
    """frac = executed warp instructions x 32 / (kernel time x lane peak): at most 1 whenever the
    instruction count is one the kernel could have issued in that time; without a record the
    fraction is null (never the algorithmic figure, which can exceed 1)."""
    sms, mhz = 152, 2070.0
    peak = sms * 128 * mhz * 1e6 / 1e12
    ms = 0.7
    # the most a kernel can issue in 0.7 ms: one warp instruction per cycle per sub-partition
    most = int(sms * 4 * mhz * 1e6 * ms * 1e-3)
    for inst in (most // 2, most):
        r = bench.fuse_roofline(1.73e9, ms, {"warp_instructions": inst, "dram_bytes_per_launch": 1},
                                peak, mhz, 0.6, 145e6, 6689.0, sms)
        assert 0 < r["frac"] <= 1.0 + 1e-9 and r["bound"] == "alu"
        assert r["algorithmic"]["lane_ops_per_s_T"] > r["achieved"]   # the uniform-march count
    r = bench.fuse_roofline(1.73e9, ms, None, peak, mhz, 0.6, 145e6, 6689.0, sms)
    assert r["frac"] is None and r["achieved"] is None and r["traffic"] is None
