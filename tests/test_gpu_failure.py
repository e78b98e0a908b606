"""Failure detection on the GPU without a fault: a bounded device wait that
runs out returns a status the host reads, and the handle stays usable."""
import numpy as np
import pytest

from paper_2604_11599_gb300.ir import Circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_bounded_wait_timeout_reaches_caller(svmod, dtype):
    """The pass kernels' tensor-core completion wait, run on an mbarrier that
    nothing arrives at (no MMA issued, a small poll limit): SV_ERR_TIMEOUT comes
    back through the control block, and the next run on the same handle is
    correct."""
    with svmod.State(6, dtype) as st:
        for polls in (0, 1, 1000):
            with pytest.raises(svmod.SVError) as e:
                st.selftest_wait(polls)
            assert e.value.status == -4  # SV_ERR_TIMEOUT
            assert "ran out" in str(e.value)
        c = Circuit(6)
        c.h(0)
        c.cx(0, 3)
        c.measure(0, 0)
        creg = st.run(c.ops, shot=5)
        a = st.amplitudes()
        want = np.zeros(64, dtype=np.complex128)
        want[9 * creg] = 1.0
        assert np.max(np.abs(a - want)) < 1e-6


def test_selftest_wait_rejects_huge_limits(svmod):
    with svmod.State(3, "c64") as st:
        with pytest.raises(svmod.SVError, match="ARG"):
            st.selftest_wait(1 << 25)
