import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Near-threshold draws of the parity comparisons (oracle margins
    |u - p0/(p0+p1)|): counted within 1e-9 and within the dtype's band, with
    the trajectories that needed a forced-outcome oracle re-run."""
    try:
        from paritylib import NEAR
    except ImportError:
        return
    if not NEAR:
        return
    tr = terminalreporter
    tr.write_sep("-", "near-threshold draws (oracle margin)")
    tr.write_line(f"{'comparison':58s} {'draws':>9s} {'<1e-9':>6s} {'<band':>6s} {'forced':>6s} {'band-mism':>9s}")
    for k in sorted(NEAR):
        d = NEAR[k]
        tr.write_line(f"{k[:58]:58s} {d['draws']:9d} {d['near_1e-9']:6d} {d['near_band']:6d} {d['forced']:6d} "
                      f"{d['mismatch_in_band']:9d}")
