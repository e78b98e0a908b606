"""CPU pins of the stabilizer-tableau rules the Clifford kernel implements:
the model's records equal the state-vector oracle's per-shot records (same
Philox draws) on random dynamic Clifford programs, and the repetition code's
closed forms hold."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import Circuit

import tableau_model as TM

BAND = 1e-9  # margins below this are near-threshold draws (counted, not compared)


def _model_shots(orc, ops, n, shots, seed=0, stream=0):
    return np.array([TM.run(ops, n, orc.uniform, seed, stream, s) for s in range(shots)], dtype=np.uint64)


@pytest.mark.parametrize("seed,n", [(1, 2), (2, 3), (3, 5), (4, 6), (5, 8)])
def test_model_matches_oracle_random_dynamic(orc, seed, n):
    c = W.random_clifford_dynamic(seed, n, n_ops=70)
    shots = 60
    got = _model_shots(orc, c.ops, n, shots, seed=3, stream=seed)
    want, _, margins = orc.run_shots(c.ops, n, shots, seed=3, stream=seed)
    ok = margins > BAND
    assert ok.mean() > 0.9
    assert np.array_equal(got[ok], want[ok])


def test_each_gate_against_oracle(orc):
    """Every gate of the set after a random Clifford prefix, each qubit then
    measured in its own random basis (Z, X or Y, by appended basis changes):
    a wrong sign or bit rule in any one conjugation changes some record
    (a sign on a mixed X/Y stabiliser shows only in mixed-basis parities)."""
    rng = np.random.default_rng(0)
    names = ["h", "s", "sdg", "x", "y", "z", "sx", "cx", "cy", "cz", "swap"]
    for g in names:
        for trial in range(12):
            n = 3
            c = W.random_clifford(int(rng.integers(1 << 30)), n, 12)
            if g in ("cx", "cy", "cz", "swap"):
                a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
                getattr(c, g)(a, b)
            else:
                getattr(c, g)(int(rng.integers(n)))
            for q in range(n):
                basis = int(rng.integers(3))
                if basis == 1:
                    c.h(q)
                elif basis == 2:
                    c.sdg(q).h(q)
                c.measure(q, q)
            got = _model_shots(orc, c.ops, n, 24, seed=trial)
            want, _, margins = orc.run_shots(c.ops, n, 24, seed=trial)
            ok = margins > BAND
            assert np.array_equal(got[ok], want[ok]), (g, trial)


_PREP1 = {"0": [], "1": ["x"], "+": ["h"], "-": ["x", "h"], "+i": ["h", "s"], "-i": ["h", "sdg"]}


def _basis(c, q, b):
    if b == "X":
        c.h(q)
    elif b == "Y":
        c.sdg(q).h(q)


def test_gates_exhaustive_small(orc):
    """Each one-qubit gate on each of the six one-qubit stabiliser states, read
    in Z, X and Y; each two-qubit gate (both orientations) on Bell-type pairs
    (|00>+|11>, |00>-|11>, |01>+|10>, |01>-|10>) and product states, read in
    all nine basis pairs: every sign and bit rule of every conjugation is
    exercised where it decides an outcome or a parity."""
    cases = []
    for g in ("h", "s", "sdg", "x", "y", "z", "sx"):
        for prep in _PREP1.values():
            for b in "ZXY":
                c = Circuit(1)
                for p in prep:
                    getattr(c, p)(0)
                getattr(c, g)(0)
                _basis(c, 0, b)
                c.measure(0, 0)
                cases.append((c, 1))
    preps2 = [["h0", "cx01"], ["h0", "cx01", "z0"], ["h0", "cx01", "x1"], ["h0", "cx01", "x1", "z0"],
              ["h0", "s1"], ["x0", "h1"]]
    for g in ("cx", "cy", "cz", "swap"):
        for a, bq in ((0, 1), (1, 0)):
            for prep in preps2:
                for b0 in "ZXY":
                    for b1 in "ZXY":
                        c = Circuit(2)
                        for p in prep:
                            if p.startswith("cx"):
                                c.cx(int(p[2]), int(p[3]))
                            else:
                                getattr(c, p[:-1])(int(p[-1]))
                        getattr(c, g)(a, bq)
                        _basis(c, 0, b0)
                        _basis(c, 1, b1)
                        c.measure(0, 0).measure(1, 1)
                        cases.append((c, 2))
    for k, (c, n) in enumerate(cases):
        got = _model_shots(orc, c.ops, n, 8, seed=k)
        want, _, margins = orc.run_shots(c.ops, n, 8, seed=k)
        ok = margins > BAND
        assert np.array_equal(got[ok], want[ok]), k


def test_rowsum_phase_table():
    """Products of single-qubit Paulis: XY = iZ, YZ = iX, ZX = iY and the reverse
    orders give -i; the g-sum counts those exponents over all qubits."""
    X, Y, Z = (1, 0), (1, 1), (0, 1)
    assert TM.g_sum(*X, *Y) == 1 and TM.g_sum(*Y, *X) == -1
    assert TM.g_sum(*Y, *Z) == 1 and TM.g_sum(*Z, *Y) == -1
    assert TM.g_sum(*Z, *X) == 1 and TM.g_sum(*X, *Z) == -1
    for P in (X, Y, Z):
        assert TM.g_sum(*P, *P) == 0 and TM.g_sum(*P, 0, 0) == 0 and TM.g_sum(0, 0, *P) == 0
    # two qubits at once: (X Z) x (Y X) = (XY)(ZX) = (iZ)(iY) -> exponent 2
    assert TM.g_sum(0b01, 0b10, 0b11, 0b01) == 2


def test_repetition_code_closed_forms(orc):
    d = 5
    c = W.repetition_code(d, rounds=4, flip_every=1, ghz=True)
    n = 2 * d - 1
    data = (1 << d) - 1
    regs = _model_shots(orc, c.ops, n, 64, seed=1)
    vals = regs & np.uint64(data)
    assert set(vals.tolist()) <= {0, data}  # data bits all equal
    assert 10 < int((vals == data).sum()) < 54
    # last round flips qubit 3: parities 2 and 3 (bits 34, 35) set, the others clear
    synd = (regs >> np.uint64(32)) & np.uint64((1 << (d - 1)) - 1)
    assert set(synd.tolist()) == {0b1100}
    want, _, margins = orc.run_shots(c.ops, n, 16, seed=1)
    ok = margins > BAND
    assert np.array_equal(regs[:16][ok], want[ok])


def test_model_rejects_non_clifford(orc):
    c = Circuit(2)
    c.t(0)
    with pytest.raises(ValueError):
        TM.run(c.ops, 2, orc.uniform)
