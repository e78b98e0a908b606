"""Engine choice of engines.sample (host logic, no GPU)."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import engines, workloads as W
from paper_2604_11599_gb300.ir import Circuit


def test_is_clifford():
    assert engines.is_clifford(W.random_clifford_dynamic(1, 6).ops)
    assert engines.is_clifford(W.repetition_code(5, 2, ghz=True).ops)
    assert engines.is_clifford(Circuit(2).ops)
    for g in ("t", "tdg"):
        c = Circuit(2)
        c.h(0)
        getattr(c, g)(1)
        assert not engines.is_clifford(c.ops)
    c = Circuit(2)
    c.rx(0, np.pi / 2)  # Clifford up to phase, but not in the gate set
    assert not engines.is_clifford(c.ops)
    c = Circuit(2)
    c.dense([0, 1], np.eye(4))
    assert not engines.is_clifford(c.ops)
    c = Circuit(3)
    c.cond(1, 1, lambda: c.ch(0, 1))  # a non-Clifford gate inside a branch counts
    assert not engines.is_clifford(c.ops)


def test_choose():
    clif = W.random_clifford_dynamic(2, 40).ops
    assert engines.choose(clif, 40) == "clifford"
    assert engines.choose(W.plain_small().ops, 5) == "batched"
    assert engines.choose(W.layered(1, 24, layers=2).ops, 24) == "plain"
    assert engines.choose(W.layered(1, 24, layers=2).ops, 24, batch_max_n=24) == "batched"
    with pytest.raises(ValueError):
        engines.choose(W.layered(1, 36, layers=1).ops, 36)
    with pytest.raises(ValueError):
        engines.sample(W.plain_small().ops, 5, 10, engine="nope")
