"""OpenQASM 3 subset front end: lowering checked record by record against the
IR builder, and whole programs against what the mathematics fixes (oracle)."""
import math

import numpy as np
import pytest

from paper_2604_11599_gb300 import qasm
from paper_2604_11599_gb300.ir import Circuit, Gate, Kind, Param


def same_ops(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.tobytes() == y.tobytes()


def test_gates_registers_and_broadcast():
    p = qasm.lower("""
        OPENQASM 3.0;
        include "stdgates.inc";
        qubit[3] q;
        qubit a;
        h q;               // broadcast over the register
        cx q[0], a;
        rz(pi / 4) q[2];
        U(0.1, 0.2, 0.3) a;
        swap q[1], q[2];
    """)
    c = Circuit(4)
    for k in range(3):
        c.h(k)
    c.cx(0, 3)
    c.rz(2, math.pi / 4)
    c.u(3, 0.1, 0.2, 0.3)
    c.swap(1, 2)
    assert p.n_qubits == 4 and p.qregs == {"q": (0, 3), "a": (3, 1)}
    same_ops(p.ops, c.ops)


def test_inputs_are_runtime_parameters():
    p = qasm.lower("""
        qubit[2] q;
        input float[64] theta;
        input angle phi;
        rx(2 * theta) q[0];
        ry(-phi / 2) q[1];
        crz(theta) q[0], q[1];
    """)
    assert p.params == {"theta": 0, "phi": 1}
    c = Circuit(2)
    c.rx(0, Param(0, 2.0))
    c.ry(1, Param(1, -0.5))
    c.crz(0, 1, Param(0, 1.0))
    same_ops(p.ops, c.ops)
    with pytest.raises(qasm.QasmError, match="offset"):
        qasm.lower("qubit q; input float t; rx(t + 1) q;")
    with pytest.raises(qasm.QasmError):
        qasm.lower("qubit q; input float t; rx(t * t) q;")


def test_measure_reset_if_else():
    p = qasm.lower("""
        qubit[2] q;
        bit[2] c;
        h q[0];
        c[0] = measure q[0];
        measure q[1] -> c[1];
        if (c[0] == 1) { x q[0]; } else { z q[1]; }
        if (c == 2) x q[1];
        if (!c[1]) { reset q[1]; }
    """)
    c = Circuit(2)
    c.h(0)
    c.measure(0, 0)
    c.measure(1, 1)
    c.cond(1, 1, lambda: c.x(0), lambda: c.z(1))
    c.cond(3, 2, lambda: c.x(1))
    c.cond(2, 2, lambda: None, lambda: c.reset(1))
    same_ops(p.ops, c.ops)
    assert p.cregs == {"c": (0, 2)} and p.n_bits == 2


def test_loops_bounded_or_unrolled():
    p = qasm.lower("""
        qubit[3] q;
        bit r;
        for uint i in [0:2] { h q[i]; }      // uses i: unrolled (ranges include their end)
        for int[32] k in [0:3] {             // does not: one LOOP record of 4 iterations
            reset q[0];
            r = measure q[0];
        }
        for i in {2, 0} x q[i];
    """)
    c = Circuit(3)
    for k in range(3):
        c.h(k)
    c.loop(4, lambda: (c.reset(0), c.measure(0, 0)))
    c.x(2)
    c.x(0)
    same_ops(p.ops, c.ops)
    with pytest.raises(qasm.QasmError, match="while"):
        qasm.lower("qubit q; bit b; while (b == 0) { b = measure q; }")


def test_modifiers_and_gate_definitions(orc):
    p = qasm.lower("""
        qubit[3] q;
        gate bell a, b { h a; cx a, b; }
        gate rot(t) a { rz(t) a; ry(t / 2) a; }
        bell q[0], q[1];
        rot(0.7) q[2];
        ctrl @ x q[2], q[0];
        inv @ s q[1];
        inv @ rx(0.3) q[0];
        pow(2) @ t q[2];
        ctrl(2) @ x q[0], q[1], q[2];
        ctrl @ h q[1], q[2];
    """)
    c = Circuit(3)
    c.h(0); c.cx(0, 1)
    c.rz(2, 0.7); c.ry(2, 0.35)
    c.cx(2, 0)
    c.sdg(1)
    c.rx(0, -0.3)
    c.t(2); c.t(2)
    tof = np.eye(8, dtype=complex)
    tof[[3, 7]] = tof[[7, 3]]  # controls q0, q1 (local bits 0, 1), target q2 (bit 2)
    c.dense([0, 1, 2], tof)
    c.ch(1, 2)
    a = orc.run(p.ops, 3, pool=p.pool).psi
    b = orc.run(c.ops, 3, pool=c.pool).psi
    assert np.max(np.abs(a - b)) < 1e-12


def test_conditional_reset_program_ends_in_zero(orc):
    """Measure |+>, flip on outcome 1: |0> on every shot (Fig. 2 pattern)."""
    p = qasm.lower("""
        OPENQASM 3;
        qubit q;
        bit c;
        h q;
        c = measure q;
        if (c == 1) { x q; }
    """)
    ones = 0
    for shot in range(64):
        t = orc.run(p.ops, 1, shot=shot)
        assert abs(t.psi[0]) == pytest.approx(1.0) and abs(t.psi[1]) < 1e-15
        ones += t.creg & 1
    assert 10 < ones < 54


def test_teleportation_program(orc):
    """Teleport U(t, f, l)|0> from q0 to q2 with feed-forward corrections, then undo
    U on q2: q2 is |0> with probability 1 on every shot."""
    th, ph, la = 1.1, 0.4, -0.9
    p = qasm.lower(f"""
        qubit[3] q;
        bit[2] m;
        U({th}, {ph}, {la}) q[0];
        h q[1];
        cx q[1], q[2];
        cx q[0], q[1];
        h q[0];
        m[0] = measure q[0];
        m[1] = measure q[1];
        if (m[1] == 1) x q[2];
        if (m[0] == 1) z q[2];
        inv @ U({th}, {ph}, {la}) q[2];
    """)
    for shot in range(16):
        psi = orc.run(p.ops, 3, shot=shot).psi.reshape(2, 4)
        assert np.sum(np.abs(psi[1]) ** 2) < 1e-24


def test_errors_name_the_line():
    with pytest.raises(qasm.QasmError, match="line 3"):
        qasm.lower("qubit q;\nh q;\nfoo q;\n")
    with pytest.raises(qasm.QasmError, match="unknown qubit"):
        qasm.lower("qubit q; h r;")
    with pytest.raises(qasm.QasmError, match="outside"):
        qasm.lower("qubit[2] q; h q[2];")
    with pytest.raises(qasm.QasmError, match="64"):
        qasm.lower("qubit q; bit[40] a; bit[30] b;")


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_qasm_program_on_the_gpu(orc, dtype):
    """A lowered dynamic program (inputs, loop, if/else, reset) runs on the GPU in
    parity with the oracle."""
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv
    from paritylib import compare_run

    p = qasm.lower("""
        qubit[12] q;
        bit[4] c;
        input float theta;
        for uint i in [0:11] { ry(theta) q[i]; }
        for uint i in [0:10] { cx q[i], q[i + 1]; }
        c[0] = measure q[3];
        if (c[0] == 1) { x q[3]; rz(2 * theta) q[7]; } else { h q[5]; }
        for uint k in [0:2] { reset q[9]; ry(theta) q[9]; c[1] = measure q[9]; }
        ctrl @ rx(theta) q[1], q[10];
        c[2] = measure q[10];
        if (c == 5) swap q[0], q[11];
    """)
    with sv.State(p.n_qubits, dtype) as st:
        for shot in range(6):
            compare_run(st, orc, p.ops, p.n_qubits, dtype, params=[0.9], seed=2, shot=shot)
