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
    c.cond(2, 0, lambda: c.reset(1))  # !c[1]: the bit tested for 0
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


def _apply(psi, u, qubits):
    """u (local index bit r <-> qubits[r]) applied to a little-endian state."""
    n = int(round(math.log2(psi.size)))
    k = len(qubits)
    out = np.zeros_like(psi)
    for i in range(psi.size):
        loc = sum(((i >> q) & 1) << r for r, q in enumerate(qubits))
        rest = i & ~sum(1 << q for q in qubits)
        for j in range(1 << k):
            tgt = rest | sum(((j >> r) & 1) << q for r, q in enumerate(qubits))
            out[tgt] += u[j, loc] * psi[i]
    assert n >= k
    return out


_PREP = "OPENQASM 3; qubit[3] q; ry(0.7) q[0]; rx(1.1) q[1]; u(0.4, 0.9, -0.3) q[2]; cx q[0], q[2]; "


def _pauli(c):
    return {"X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
            "Z": np.array([[1, 0], [0, -1]])}[c].astype(np.complex128)


@pytest.mark.parametrize("stmt,u,qubits", [
    ("rzz(0.8) q[0], q[2];", None, (0, 2)),
    ("rxx(0.8) q[1], q[0];", None, (1, 0)),
    ("ryy(0.8) q[2], q[1];", None, (2, 1)),
    ("rzx(0.8) q[0], q[1];", None, (0, 1)),
    ("inv @ rzz(0.8) q[0], q[2];", "inv", (0, 2)),
    ("sxdg q[1];", "sxdg", (1,)),
    ("negctrl @ x q[0], q[1];", "negx", (0, 1)),
    ("negctrl @ ctrl @ x q[2], q[0], q[1];", "negctrl-ctrl-x", (2, 0, 1)),
    ("ctrl @ gphase(0.6) q[1];", "cphase", (1,)),
    ("gphase(0.6);", "global", ()),
])
def test_extra_gates_and_modifiers_against_matrices(orc, stmt, u, qubits):
    """Each construct against its matrix applied to the state the prefix prepares."""
    psi0 = orc.run(qasm.lower(_PREP).ops, 3).psi
    prog = qasm.lower(_PREP + stmt)
    got = orc.run(prog.ops, 3, pool=prog.pool).psi
    t = 0.8
    name = stmt.split("(")[0].split()[0]
    if u is None or u == "inv":
        if u == "inv":
            t, name = -t, "rzz"
        pa, pb = {"rzz": "ZZ", "rxx": "XX", "ryy": "YY", "rzx": "ZX"}[name]
        pp = np.kron(_pauli(pb), _pauli(pa))  # local bit 0 <-> first qubit
        m = math.cos(t / 2) * np.eye(4) - 1j * math.sin(t / 2) * pp
        want = _apply(psi0, m, qubits)
    elif u == "sxdg":
        sx = np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]) / 2
        want = _apply(psi0, sx.conj().T, qubits)
    elif u == "negx":  # X on the target when the control is |0>
        m = np.eye(4, dtype=np.complex128)
        m[[0, 2]] = m[[2, 0]]
        want = _apply(psi0, m, qubits)
    elif u == "negctrl-ctrl-x":  # X on q[1] when q[2] = 0 and q[0] = 1
        m = np.eye(8, dtype=np.complex128)
        a, b = 0b010, 0b110  # local bits: r0 = q2 (0), r1 = q0 (1), r2 = target
        m[[a, b]] = m[[b, a]]
        want = _apply(psi0, m, qubits)
    elif u == "cphase":
        want = _apply(psi0, np.diag([1, np.exp(0.6j)]), qubits)
    else:
        want = np.exp(0.6j) * psi0
    assert np.max(np.abs(got - want)) < 1e-12


_GDEF = ("gate g(x) a, b { s a; h b; cx a, b; rz(x) b; sx a; swap a, b; t b; u(0.3, 0.2, 0.1) a; "
         "ctrl @ ry(0.4) b, a; } ")


def test_inverse_of_a_user_gate(orc):
    """g then inv @ g gives back the prepared state (records reversed, each inverted)."""
    src = _PREP.replace("qubit[3] q; ", "qubit[3] q; " + _GDEF)
    psi0 = orc.run(qasm.lower(src).ops, 3).psi
    prog = qasm.lower(src + "g(0.7) q[0], q[2]; inv @ g(0.7) q[0], q[2];")
    psi = orc.run(prog.ops, 3, pool=prog.pool).psi
    assert np.max(np.abs(psi - psi0)) < 1e-12
    prog = qasm.lower(src + "inv @ g(0.7) q[2], q[1]; g(0.7) q[2], q[1];")  # the other order too
    assert np.max(np.abs(orc.run(prog.ops, 3, pool=prog.pool).psi - psi0)) < 1e-12


def test_controlled_user_gate(orc):
    """ctrl @ g equals diag(I, U) with U, g's unitary, assembled column by column."""
    head = "OPENQASM 3; qubit[3] q; " + _GDEF
    u = np.zeros((4, 4), dtype=np.complex128)
    for col in range(4):  # local bit 0 <-> q[1], bit 1 <-> q[2]
        prep = "".join(f"x q[{1 + r}]; " for r in range(2) if (col >> r) & 1)
        prog = qasm.lower(head + prep + "g(0.7) q[1], q[2];")
        psi = orc.run(prog.ops, 3, pool=prog.pool).psi
        for row in range(4):
            u[row, col] = psi[(row & 1) << 1 | (row >> 1) << 2]
    cu = np.eye(8, dtype=np.complex128)  # local bit 0 <-> q[0] (control), bits 1, 2 <-> q[1], q[2]
    for a in range(4):
        for b in range(4):
            cu[1 | a << 1, 1 | b << 1] = u[a, b]
    psi0 = orc.run(qasm.lower(_PREP).ops, 3).psi
    prog = qasm.lower(_PREP.replace("qubit[3] q; ", "qubit[3] q; " + _GDEF) + "ctrl @ g(0.7) q[0], q[1], q[2];")
    got = orc.run(prog.ops, 3, pool=prog.pool).psi
    assert np.max(np.abs(got - _apply(psi0, cu, (0, 1, 2)))) < 1e-12


def test_measure_forms_slices_and_delay(orc):
    p = qasm.lower("OPENQASM 3; qubit[4] q; x q[1:3]; delay[20ns] q; bit[2] c = measure q[0:1]; measure q[3];")
    meas = p.ops[p.ops["kind"] == int(Kind.MEASURE)]
    assert [(int(o["q"][0]), int(o["cbit"])) for o in meas] == [(0, 0), (1, 1), (3, qasm.HIDDEN_BIT)]
    r = orc.run(p.ops, 4)
    assert r.creg == 0b10 | (1 << qasm.HIDDEN_BIT)
    p = qasm.lower("OPENQASM 3; qubit[4] q; x q[3:-2:0];")  # 3, 1
    assert [int(o["q"][0]) for o in p.ops] == [3, 1]
    with pytest.raises(qasm.QasmError):
        qasm.lower("OPENQASM 3; qubit[2] q; x q[0:5];")


@pytest.mark.parametrize("cond,f", [
    ("c[0] && !c[1]", lambda a, b: a and not b),
    ("c[0] == 1 && c[1] == true", lambda a, b: a and b),
    ("c[0] || c[1]", lambda a, b: a or b),
    ("!(c[0] || c[1])", lambda a, b: not (a or b)),
    ("!(c[0] && c[1])", lambda a, b: not (a and b)),
    ("c == 2", lambda a, b: (not a) and b),
    ("c != 3", lambda a, b: not (a and b)),
    ("(c[0]) && (c[1] == 0) || c == 2", lambda a, b: (a and not b) or ((not a) and b)),
    ("c[0] && !c[0]", lambda a, b: False),
    ("c[1] != 1", lambda a, b: not b),
])
def test_compound_conditions(orc, cond, f):
    """Two bits drawn uniformly decide an X on a third qubit through the condition:
    its readout equals the formula on every shot, for every one of the four records."""
    src = ("OPENQASM 3; qubit[3] q; bit[2] c; bit r; h q[0]; h q[1]; c = measure q[0:1]; "
           f"if ({cond}) {{ x q[2]; }} else {{ }} r = measure q[2];")
    prog = qasm.lower(src)
    regs, _, _ = orc.run_shots(prog.ops, 3, 64, seed=5)
    seen = set()
    for v in regs.tolist():
        a, b, r = v & 1, (v >> 1) & 1, (v >> 2) & 1
        seen.add((a, b))
        assert r == int(bool(f(a, b))), (cond, a, b, r)
    assert len(seen) == 4


def test_subroutines_inline_to_the_written_out_program(orc):
    """def subroutines (qubit, bit, float arguments; a returned measurement) lower
    to exactly the records of the same program written out by hand."""
    with_defs = qasm.lower("""OPENQASM 3; qubit[4] q; bit[3] c; input float t;
        def parity(qubit a, qubit b, qubit anc) -> bit { reset anc; cx a, anc; cx b, anc; return measure anc; }
        def flipif(qubit tq, bit s) { if (s) { x tq; } }
        def rot(qubit tq, float th) { rx(th) tq; rz(th / 2) tq; }
        def layer(qubit[2] r, float th) { for int i in [0:1] { rot(r[i], th); } cx r[0], r[1]; }
        h q[0]; h q[1];
        c[0] = parity(q[0], q[1], q[3]);
        flipif(q[2], c[0]);
        layer(q[1:2], t);
        c[1] = measure q[2];
        parity(q[1], q[2], q[3]);
        c[2] = parity(q[0], q[2], q[3]);
    """)
    written = qasm.lower("""OPENQASM 3; qubit[4] q; bit[3] c; input float t;
        h q[0]; h q[1];
        reset q[3]; cx q[0], q[3]; cx q[1], q[3]; c[0] = measure q[3];
        if (c[0]) { x q[2]; }
        rx(t) q[1]; rz(t / 2) q[1]; rx(t) q[2]; rz(t / 2) q[2]; cx q[1], q[2];
        c[1] = measure q[2];
        reset q[3]; cx q[1], q[3]; cx q[2], q[3]; measure q[3];
        reset q[3]; cx q[0], q[3]; cx q[2], q[3]; c[2] = measure q[3];
    """)
    same_ops(with_defs.ops, written.ops)
    r = orc.run(with_defs.ops, 4, params=[0.3], seed=1)
    assert r.status == 0


@pytest.mark.parametrize("src,msg", [
    ("def f(qubit a) -> bit { return measure a; } qubit[2] q; f(q);", "takes 1 qubits"),
    ("def f(qubit a) { return measure a; } qubit q; f(q);", "return outside"),
    ("def f(qubit a, bit s) -> bit { if (s) { return measure a; } } qubit q; bit[2] c; c[0] = f(q, c[1]);",
     "top of a subroutine"),
    ("def f(qubit a) { bit b; } qubit q; f(q);", "classical declarations"),
    ("def f(qubit a) { f(a); } qubit q; f(q);", "nested too deeply"),
    ("def f(qubit a) { x a; } qubit q; bit c; c = f(q);", "returns nothing"),
    ("def f(bit[2] b) { } qubit q; bit[4] c; f(c[0:2:2]);", "consecutive bits"),
])
def test_subroutine_errors(src, msg):
    with pytest.raises(qasm.QasmError, match=msg):
        qasm.lower("OPENQASM 3; " + src)


def test_extra_forms_lower_to_records():
    p = qasm.lower("OPENQASM 3; qubit[3] q; negctrl(2) @ x q[0], q[1], q[2];")
    kinds = [int(k) for k in p.ops["kind"]]
    assert kinds == [int(Kind.GATE)] * 2 + [int(Kind.DENSE)] + [int(Kind.GATE)] * 2
    assert [int(g) for g in p.ops["gate"][[0, 1, 3, 4]]] == [int(Gate.X)] * 4
    p = qasm.lower("OPENQASM 3; input float t; qubit[2] q; rzz(t) q[0], q[1];")
    rz = p.ops[p.ops["gate"] == int(Gate.RZ)]
    assert len(rz) == 1 and int(rz[0]["pidx"][0]) == 0 and int(rz[0]["q"][0]) == 1
    with pytest.raises(qasm.QasmError):
        qasm.lower("OPENQASM 3; qubit[2] q; gphase(0.1) q[0];")  # gphase takes controls only


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
