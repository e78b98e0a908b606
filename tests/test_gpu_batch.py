"""Batched persistent launch: every trajectory's record equals the plain path's
(same seed, stream, shot) and the oracle's; uneven qubit counts share one launch."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2604_11599_gb300 import workloads as W

from paritylib import BAND

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_matches_plain_path_mixed_n(svmod, orc, dtype):
    """Sequential feed-forward + RUS circuits on 4..17 qubits (several multi-tile
    states) in one launch; records bit-exact against sv_run per trajectory."""
    ns = [3, 5, 8, 11, 13, 14, 16]
    circs = {n: W.sequential_feedforward(500 + n, n, layers=4) for n in ns}
    rng = np.random.default_rng(0)
    traj_n = rng.choice(ns, size=70)
    with svmod.Batch(dtype) as b:
        pid = {n: b.add_program(circs[n].ops, n + 1) for n in ns}
        streams = np.arange(len(traj_n), dtype=np.uint64) + 100
        shots = rng.integers(0, 1000, size=len(traj_n)).astype(np.uint64)
        got = b.run([pid[n] for n in traj_n], streams, shots, seed=7)
    for n in ns:
        idx = np.nonzero(traj_n == n)[0]
        with svmod.State(n + 1, dtype) as st:
            for i in idx:
                want = st.run(circs[n].ops, seed=7, stream_id=int(streams[i]), shot=int(shots[i]))
                assert int(got[i]) == want, (n, i)
    # and against the oracle on a few trajectories per size
    for n in ns:
        for i in np.nonzero(traj_n == n)[0][:2]:
            ref = orc.run(circs[n].ops, n + 1, seed=7, stream=int(streams[i]), shot=int(shots[i]))
            if (ref.draws["margin"] > BAND[dtype]).all():
                assert int(got[i]) == ref.creg


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_specialised_kernel_matches_generic(svmod, dtype):
    """The batch kernel specialised to the programs (sv_batch_set_jit) gives the
    generic kernel's records on a mix of sizes, and is rebuilt when a program is
    added; records of the plain path cover the new program."""
    ns = [5, 11, 13]
    circs = {n: W.sequential_feedforward(700 + n, n, layers=3) for n in ns}
    rng = np.random.default_rng(3)
    traj_n = rng.choice(ns, size=48)
    streams = np.arange(len(traj_n), dtype=np.uint64) + 9
    shots = rng.integers(0, 1000, size=len(traj_n)).astype(np.uint64)
    with svmod.Batch(dtype) as b:
        pid = {n: b.add_program(circs[n].ops, n + 1) for n in ns}
        ids = [pid[n] for n in traj_n]
        generic = b.run(ids, streams, shots, seed=3)
        b.set_jit(True)
        spec = b.run(ids, streams, shots, seed=3)
        assert b.jit_info()["specialised"]
        assert np.array_equal(generic, spec)
        extra = W.sequential_feedforward(99, 7, layers=3)
        p7 = b.add_program(extra.ops, 8)  # the next launch builds the kernel again
        got = b.run([p7] * 8, np.arange(8, dtype=np.uint64), np.arange(8, dtype=np.uint64), seed=3)
        assert b.jit_info()["specialised"]
    with svmod.State(8, dtype) as st:
        for i in range(8):
            assert int(got[i]) == st.run(extra.ops, seed=3, stream_id=i, shot=i)


def test_batch_graph_replay_and_seed(svmod):
    c = W.sequential_feedforward(9, 6, layers=3)
    with svmod.Batch("c64") as b:
        p = b.add_program(c.ops, 7)
        b.set_items([p] * 300, np.arange(300), np.zeros(300))
        b.launch(seed=1)
        r1 = b.results()
        b.launch(seed=1)
        r2 = b.results()
        b.launch(seed=2)
        r3 = b.results()
    assert np.array_equal(r1, r2)
    assert not np.array_equal(r1, r3)


def test_batch_plain_small_config_shots(svmod, orc):
    """Plain-path program (complex128, n=5) for 1,000 shots through the batched
    launch: identical records to the plain path and the oracle."""
    c = W.plain_small()
    with svmod.Batch("c128") as b:
        p = b.add_program(c.ops, 5)
        got = b.run([p] * 1000, np.zeros(1000), np.arange(1000), seed=0)
    cregs, _, margins = orc.run_shots(c.ops, 5, 1000, seed=0)
    ok = margins > BAND["c128"]
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], cregs[ok])


def test_batch_rus_success_probability(svmod):
    """The ancilla RUS loop succeeds within 4 tries with probability 1 - cos^8(theta/2)."""
    c = W.sequential_feedforward(31, 4, layers=2)
    shots = 20000
    with svmod.Batch("c64") as b:
        p = b.add_program(c.ops, 5)
        got = b.run(np.full(shots, p), np.arange(shots), np.zeros(shots), seed=3)
    ok = int(((got >> np.uint64(63)) & np.uint64(1)).sum())
    pr = 1 - math.cos(c.rus_theta / 2) ** 8
    assert stats.binomtest(ok, shots, pr).pvalue > 1e-4


def test_batch_errors(svmod):
    with svmod.Batch("c64") as b:
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            b.set_items([3], [0], [0])
        from paper_2604_11599_gb300.ir import Circuit

        c = Circuit(3)
        c.x(5)
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            b.add_program(c.ops, 3)
