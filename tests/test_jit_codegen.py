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
