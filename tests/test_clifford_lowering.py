"""Clifford path, host side: the lowering refuses what the tableaux cannot run
before any device call (non-Clifford gates, dense records, bad qubits or bits,
inconsistent lengths, unrolled programs beyond 2^24 instructions)."""
import numpy as np
import pytest

from paper_2604_11599_gb300.ir import Circuit, Kind


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


def _refused(svmod, n, ops, code):
    with pytest.raises(svmod.SVError, match=code):
        svmod.Clifford(n, ops)


def test_non_clifford_and_dense_refused(svmod):
    for g in ("t", "tdg"):
        c = Circuit(2)
        c.h(0)
        getattr(c, g)(1)
        _refused(svmod, 2, c.ops, "SV_ERR_UNSUPPORTED")
    c = Circuit(2)
    c.rx(0, 0.5)
    _refused(svmod, 2, c.ops, "SV_ERR_UNSUPPORTED")
    c = Circuit(2)
    c.dense([0, 1], np.eye(4))
    _refused(svmod, 2, c.ops, "SV_ERR_UNSUPPORTED")
    c = Circuit(2)
    c.cond(1, 1, lambda: c.ch(0, 1))  # refused inside a branch too
    _refused(svmod, 2, c.ops, "SV_ERR_UNSUPPORTED")


def test_bad_arguments_refused(svmod):
    c = Circuit(3)
    c.x(3)
    _refused(svmod, 3, c.ops, "SV_ERR_ARG")  # qubit out of range
    c = Circuit(3)
    c.cx(1, 1)
    _refused(svmod, 3, c.ops, "SV_ERR_ARG")  # one qubit twice
    for n in (0, 65):
        _refused(svmod, n, Circuit(2).ops, "SV_ERR_ARG")
    c = Circuit(2)
    c.cond(1, 1, lambda: c.x(0))
    ops = c.ops
    ops[0]["then_len"] = 5  # runs past the end
    _refused(svmod, 2, ops, "SV_ERR_ARG")
    c = Circuit(2)
    c.measure(0, 3)
    ops = c.ops
    ops[0]["cbit"] = 64
    _refused(svmod, 2, ops, "SV_ERR_ARG")


def test_unroll_limit(svmod):
    c = Circuit(2)
    c.loop(1 << 16, lambda: c.loop(1 << 9, lambda: c.h(0)))  # 2^25 instructions
    assert int(c.ops[0]["kind"]) == int(Kind.LOOP)
    _refused(svmod, 2, c.ops, "SV_ERR_UNSUPPORTED")


def test_valid_programs_pass_the_lowering(svmod):
    """Large valid programs (63 and 64 qubits, feed-forward, loops) pass the
    size check and the lowering; without a GPU the first device call fails."""
    import torch

    from paper_2604_11599_gb300 import workloads as W

    if torch.cuda.is_available():
        pytest.skip("with a GPU the handle is created (covered by the GPU tests)")
    for c, n in ((W.repetition_code(32, 10, flip_every=1, ghz=True), 63),
                 (W.random_clifford_dynamic(21, 64, n_ops=150), 64)):
        with pytest.raises(svmod.SVError, match="SV_ERR_CUDA"):
            svmod.Clifford(n, c.ops)
