"""The pass specialiser generates code that NVRTC compiles for sm_103a (host only, no GPU)."""
import pytest

from paper_2604_11599_gb300 import workloads as W


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_every_gate_and_dense_compiles(svmod, dtype):
    c = W.random_static(11, 14, 80, dense_k=3, params=3)
    svmod.jit_check(c.ops, 14, dtype, pool=c.pool)
    c = W.random_static(12, 13, 60, dense_k=4)
    svmod.jit_check(c.ops, 13, dtype, pool=c.pool)


def test_dynamic_program_with_predicated_gates_compiles(svmod):
    c = W.random_dynamic(5, 16, n_ops=60)
    svmod.jit_check(c.ops, 16, "c64")


def test_compile_errors_are_reported(svmod):
    from paper_2604_11599_gb300.ir import Circuit

    c = Circuit(3)
    c.x(7)
    with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
        svmod.jit_check(c.ops, 3, "c64")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_specialised_adjoint_kernel_compiles(svmod, dtype):
    """The adjoint kernel specialised to a program (forward stage programs in
    CTA mode, backward phi/lambda stages with every parametrised gate kind,
    shared parameters, dense two- and three-qubit gates) compiles for sm_103a;
    on the VQE ansatz its registers spill little at the kernel's CTAs per SM."""
    import re

    import numpy as np

    from paper_2604_11599_gb300.ir import Circuit, Gate, Param

    n = 6
    r = np.random.default_rng(5)
    c = Circuit(n)
    kinds = [Gate.RX, Gate.RY, Gate.RZ, Gate.P, Gate.U, Gate.CRX, Gate.CRY, Gate.CRZ, Gate.CP, Gate.CU]
    for g in kinds:
        qs = [int(v) for v in r.choice(n, size=2 if g.name.startswith("C") else 1, replace=False)]
        angs = [Param(int(r.integers(4)), 1.0) for _ in range(3 if g in (Gate.U, Gate.CU) else 1)]
        c.gate(g, qs, angs)
        c.gate(Gate.CX, [int(v) for v in r.choice(n, size=2, replace=False)])
    for k in (2, 3):
        u, _ = np.linalg.qr(r.normal(size=(1 << k, 1 << k)) + 1j * r.normal(size=(1 << k, 1 << k)))
        c.dense([int(v) for v in r.choice(n, size=k, replace=False)], u)
    log = svmod.jit_check_adjoint(c.ops, n, dtype, pool=c.pool)
    assert "sv_jit_adjoint" in log
    log = svmod.jit_check_adjoint(W.hea(8, 2).ops, 8, dtype)
    spills = [int(v) for v in re.findall(r"(\d+) bytes spill stores", log)]
    assert spills and max(spills) <= 512, log


def test_specialised_batch_kernel_compiles(svmod):
    """The batched kernel specialised to several programs (each program's
    passes as non-inlined stage functions, numbered consecutively) compiles
    for sm_103a, for programs with measurement, feed-forward and loops."""
    progs = [(W.sequential_feedforward(40 + n, n, layers=2).ops, n + 1) for n in (5, 12)]
    log = svmod.jit_check_batch(progs, "c64")
    assert "sv_jit_batch" in log
    with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
        svmod.jit_check_batch([], "c64")
