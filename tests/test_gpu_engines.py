"""engines.sample on the GPU: each engine it picks gives the records of that
engine's own per-shot call."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import engines, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


def test_auto_engines_match_their_own_calls(svmod):
    c = W.random_clifford_dynamic(5, 10, n_ops=60)
    regs, info = engines.sample(c.ops, 10, 200, seed=1)
    assert info["engine"] == "clifford"
    with svmod.Clifford(10, c.ops) as h:
        assert np.array_equal(regs, h.sample(200, seed=1))
    p = W.plain_small(seed=6)
    regs, info = engines.sample(p.ops, 5, 300, dtype="c128", seed=2)
    assert info["engine"] == "batched" and info["paths"] <= 32
    with svmod.Batch("c128") as b:
        pid = b.add_program(p.ops, 5)
        assert np.array_equal(regs, b.run(np.full(300, pid), np.zeros(300), np.arange(300), seed=2))
    L = W.layered(3, 22, layers=4)
    regs, info = engines.sample(L.ops, 22, 16, seed=3)
    assert info["engine"] == "plain"
    with svmod.State(22, "c64") as st:
        want, _ = st.sample(L.ops, 16, seed=3)
    assert np.array_equal(regs, want)
