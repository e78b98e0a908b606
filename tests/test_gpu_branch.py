"""Shot branching: every shot's record equals the record its own trajectory
gives (same engine, same seed, stream and shot), bit for bit, while only one
trajectory per distinct outcome path runs; and the records agree with the
oracle's per-shot records away from the near-threshold band."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import Circuit

from paritylib import BAND

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_plain_branched_equals_per_shot(svmod, orc, dtype):
    """The n=5 plain-path program (a measure every 8 ops into its own creg bit,
    conditional reset and a 2-bit if-else after each): 1,000 shots."""
    c = W.plain_small()
    shots = 1000
    with svmod.State(5, dtype) as st:
        want, _ = st.sample(c.ops, shots, seed=0)
        got, stats = st.sample_branched(c.ops, shots, seed=0)
    assert np.array_equal(got, want)
    # each measure writes its own bit, so the register names the outcome path
    assert stats["paths"] == len(np.unique(want))
    assert stats["shots"] == shots and stats["paths"] < shots // 10
    assert stats["levels"] <= stats["max_draws"] + 1
    cregs, _, margins = orc.run_shots(c.ops, 5, shots, seed=0)
    ok = margins > BAND[dtype]
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], cregs[ok])


@pytest.mark.parametrize("n", [14, 20])
def test_plain_branched_multi_tile(svmod, n):
    """Multi-tile states with the specialised pass kernels, loops and resets:
    a random dynamic circuit and the feed-forward + repeat-until-success one."""
    for c, nq in ((W.random_dynamic(40 + n, n, n_ops=70), n), (W.sequential_feedforward(60 + n, n - 1, layers=2), n)):
        with svmod.State(nq, "c64") as st:
            st.set_jit(True)
            want, _ = st.sample(c.ops, 96, seed=5, stream_id=3)
            got, stats = st.sample_branched(c.ops, 96, seed=5, stream_id=3)
        assert np.array_equal(got, want)
        assert 1 <= stats["paths"] <= 96


def test_plain_branched_edges(svmod):
    c = Circuit(3)
    c.h(0).cx(0, 1)
    with svmod.State(3, "c64") as st:
        got, stats = st.sample_branched(c.ops, 7)  # no draws: one path
        assert np.array_equal(got, np.zeros(7, dtype=np.uint64)) and stats["paths"] == 1
        got, stats = st.sample_branched(c.ops, 0)
        assert got.size == 0 and stats["paths"] == 0
    g = W.ghz(4)
    g.measure(0, 0).measure(1, 1).measure(2, 2).measure(3, 3)
    with svmod.State(4, "c128") as st:
        got, stats = st.sample_branched(g.ops, 4000, seed=9)
        want, _ = st.sample(g.ops, 4000, seed=9)
    assert np.array_equal(got, want)
    # GHZ: all-zero or all-one, and only the first draw is random
    assert set(np.unique(got).tolist()) <= {0, 15} and stats["paths"] == 2
    assert abs((got == 15).mean() - 0.5) < 0.05


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_branched_equals_per_shot(svmod, dtype):
    """Several requests (programs of 4..16 qubits, their own streams and shot
    counts) in one call: records equal sv_batch_run's per-shot records."""
    ns = [4, 7, 12, 16]
    circs = {n: W.sequential_feedforward(700 + n, n, layers=3) for n in ns}
    rng = np.random.default_rng(1)
    with svmod.Batch(dtype) as b:
        pid = {n: b.add_program(circs[n].ops, n + 1) for n in ns}
        small = b.add_program(W.plain_small(seed=4).ops, 5)
        reqs = [(pid[n], 50 + i, int(rng.integers(1, 400))) for i, n in enumerate(ns)]
        reqs += [(small, 99, 1500), (pid[4], 51, 0)]
        got, stats = b.sample_branched([r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs], seed=11)
        assert got.size == sum(r[2] for r in reqs) == stats["shots"]
        k = 0
        for p, s, nshots in reqs:
            want = b.run(np.full(nshots, p), np.full(nshots, s), np.arange(nshots), seed=11)
            assert np.array_equal(got[k: k + nshots], want), (p, s)
            k += nshots
    # one path per distinct outcome sequence: at most one per shot, and the
    # 1,500-shot n=5 request contributes at most 2^5
    assert 0 < stats["paths"] <= stats["shots"] - 1500 + 32


def test_batch_branched_many_shots(svmod, orc):
    """10^5 shots of the n=5 program: a sampled subset against per-shot runs
    and the oracle; far fewer trajectories than shots."""
    c = W.plain_small()
    shots = 100_000
    with svmod.Batch("c128") as b:
        p = b.add_program(c.ops, 5)
        got, stats = b.sample_branched([p], [0], [shots], seed=0)
        pick = np.random.default_rng(2).choice(shots, size=512, replace=False)
        want = b.run(np.full(pick.size, p), np.zeros(pick.size), pick.astype(np.uint64), seed=0)
    assert np.array_equal(got[pick], want)
    assert stats["paths"] <= 2 ** stats["max_draws"] and stats["paths"] < 200
    cregs, _, margins = orc.run_shots(c.ops, 5, 300, seed=0)
    ok = margins > BAND["c128"]
    assert np.array_equal(got[:300][ok], cregs[ok])
