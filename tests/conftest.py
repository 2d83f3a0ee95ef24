"""Test configuration: the `gpu` marker and shared fixtures.

Tests marked `gpu` need a CUDA device and the compiled CUDA library; all
others run on the CPU (oracle pins, host-side argument checks, symbol
exports, multi-process host logic).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the compiled CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth_mod():
    import synth
    synth.build()
    return synth


def pytest_terminal_summary(terminalreporter):
    """Report the oracle-flagged (ambiguous) fraction of every fused-depth comparison."""
    try:
        from gpu_util import AMBIGUOUS_LOG, MAX_AMBIGUOUS
    except ImportError:
        return
    if not AMBIGUOUS_LOG:
        return
    flagged = sum(a for _, a, _ in AMBIGUOUS_LOG)
    total = sum(n for _, _, n in AMBIGUOUS_LOG)
    worst = max(AMBIGUOUS_LOG, key=lambda r: r[1] / max(r[2], 1))
    terminalreporter.write_line(
        f"fused-depth comparisons: {len(AMBIGUOUS_LOG)}, flagged ambiguous {flagged} of {total} px "
        f"({flagged / max(total, 1):.2e}); worst {worst[1]}/{worst[2]} ({worst[1] / max(worst[2], 1):.2e}) in "
        f"{worst[0]}; a case fails above {MAX_AMBIGUOUS:g}")
