"""Clifford fast path (stabilizer tableaux, one warp per shot): records equal
the oracle's per-shot records away from the near-threshold band, equal the
CPU tableau model at 64 qubits (beyond the state vector), and obey the
repetition code's and GHZ's closed forms."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import Circuit

import tableau_model as TM

pytestmark = pytest.mark.gpu
BAND = 1e-9


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


@pytest.mark.parametrize("seed,n", [(11, 2), (12, 5), (13, 8), (14, 12)])
def test_clifford_vs_oracle(svmod, orc, seed, n):
    c = W.random_clifford_dynamic(seed, n, n_ops=90)
    shots = 120
    with svmod.Clifford(n, c.ops) as cl:
        got = cl.sample(shots, seed=4, stream_id=seed)
    want, _, margins = orc.run_shots(c.ops, n, shots, seed=4, stream=seed)
    ok = margins > BAND
    assert ok.mean() > 0.9
    assert np.array_equal(got[ok], want[ok])
    # and the state-vector engine on the GPU, away from the same ties
    with svmod.State(n, "c128") as st:
        sv_regs, _ = st.sample(c.ops, shots, seed=4, stream_id=seed)
    assert np.array_equal(got[ok], sv_regs[ok])


def test_clifford_vs_model_64_qubits(svmod, orc):
    """64 qubits (2^64 amplitudes: no state vector): against the CPU tableau model."""
    for seed in (21, 22):
        c = W.random_clifford_dynamic(seed, 64, n_ops=150)
        with svmod.Clifford(64, c.ops) as cl:
            got = cl.sample(24, seed=1, stream_id=seed)
        want = np.array([TM.run(c.ops, 64, orc.uniform, 1, seed, s) for s in range(24)], dtype=np.uint64)
        assert np.array_equal(got, want)


def test_repetition_code_closed_forms(svmod):
    d, rounds = 32, 6
    c = W.repetition_code(d, rounds, flip_every=1, ghz=True)
    with svmod.Clifford(2 * d - 1, c.ops) as cl:
        regs = cl.sample(100_000, seed=2)
        again = cl.sample(1000, seed=2, shot0=500)
    data = np.uint64((1 << d) - 1)
    vals = regs & data
    assert set(np.unique(vals).tolist()) <= {0, int(data)}
    assert abs(float((vals == data).mean()) - 0.5) < 0.01
    last = (rounds - 1) % d  # the last round's flip and its two parities
    want_synd = (1 << (last - 1)) | (1 << last) if 0 < last < d - 1 else (1 if last == 0 else 1 << (d - 2))
    synd = (regs >> np.uint64(32)) & np.uint64((1 << (d - 1)) - 1)
    assert set(np.unique(synd).tolist()) == {want_synd}
    assert np.array_equal(again, regs[500:1500])


def test_ghz64_parities(svmod):
    """GHZ on 64 qubits: Z readout all equal; X readout has even parity (the
    stabiliser X...X has eigenvalue +1); after S on qubits 0 and 1 the group
    holds Y_0 Y_1 X...X and Z_0 Z_1, whose product is -X...X, so the X readout
    has odd parity (a sign rule error shows here)."""
    n = 64
    g = W.ghz(n)
    z = Circuit(n)
    z._recs = list(g._recs)
    for q in range(n):
        z.measure(q, q)
    x = Circuit(n)
    x._recs = list(g._recs)
    for q in range(n):
        x.h(q).measure(q, q)
    y = Circuit(n)
    y._recs = list(g._recs)
    y.s(0).s(1)
    for q in range(n):
        y.h(q).measure(q, q)
    with svmod.Clifford(n, z.ops) as cl:
        rz = cl.sample(4000, seed=3)
    assert set(np.unique(rz).tolist()) <= {0, (1 << 64) - 1}
    for circ, want in ((x, 0), (y, 1)):
        with svmod.Clifford(n, circ.ops) as cl:
            r = cl.sample(4000, seed=3)
        par = np.array([bin(int(v)).count("1") & 1 for v in r])
        assert (par == want).all()
        assert len(np.unique(r)) > 1000  # outcomes themselves are random


def test_clifford_errors(svmod):
    c = Circuit(2)
    c.t(0)
    with pytest.raises(svmod.SVError, match="SV_ERR_UNSUPPORTED"):
        svmod.Clifford(2, c.ops)
    with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
        svmod.Clifford(65, Circuit(2).ops)
    with svmod.Clifford(3, Circuit(3).ops) as cl:  # empty program
        assert np.array_equal(cl.sample(5), np.zeros(5, dtype=np.uint64))
        assert cl.sample(0).size == 0
