"""Noise by trajectories (channels lowered into the IR), pinned on the oracle:
each channel's flip probabilities against their closed forms, the readout
error leaving the state alone, zero noise changing nothing, and structure
kept under COND and LOOP."""
import numpy as np
import pytest
from scipy import stats

from paper_2604_11599_gb300 import noise, workloads as W
from paper_2604_11599_gb300.ir import Circuit, Kind


def _ones(orc, c, n, shots, bit=0, seed=0):
    regs, _, _ = orc.run_shots(c.ops, n, shots, seed=seed)
    return int(((regs >> np.uint64(bit)) & np.uint64(1)).sum()), regs


def _check(k, shots, p):
    assert stats.binomtest(k, shots, p).pvalue > 1e-4, (k, shots, p)


def test_pauli_channel_each_component(orc):
    """px, py, pz each pinned: |0> read in Z flips under X, Y; |+> read in X
    flips under Y, Z; |+i> read in Y flips under X, Z."""
    px, py, pz = 0.1, 0.2, 0.3
    shots = 3000
    for prep, read, want in (([], [], px + py), (["h"], ["h"], py + pz), (["h", "s"], ["sdg", "h"], px + pz)):
        c = Circuit(2)
        for g in prep:
            getattr(c, g)(0)
        noise.pauli_channel(c, 0, px, py, pz, anc=1)
        for g in read:
            getattr(c, g)(0)
        c.measure(0, 0)
        k, _ = _ones(orc, c, 2, shots, seed=len(prep))
        _check(k, shots, want)


def test_depolarize_rate(orc):
    c = Circuit(2)
    noise.depolarize(c, 0, 0.3, anc=1)
    c.measure(0, 0)
    k, _ = _ones(orc, c, 2, 3000, seed=5)
    _check(k, 3000, 0.2)


def test_readout_error_keeps_state(orc):
    """The first readout of |1> is flipped with p; a second, noiseless readout
    of the same qubit always sees 1 (the state is the true post-measurement one)."""
    c = Circuit(2)
    c.x(0)
    noise.noisy_measure(c, 0, 0, 0.25, anc=1)
    c.measure(0, 1)
    k, regs = _ones(orc, c, 2, 3000, seed=6)
    _check(3000 - k, 3000, 0.25)
    assert ((regs >> np.uint64(1)) & np.uint64(1)).all()


def test_noisy_reset_rate(orc):
    c = Circuit(2)
    c.h(0)
    noise.noisy_reset(c, 0, 0.2, anc=1)
    c.measure(0, 0)
    k, _ = _ones(orc, c, 2, 3000, seed=7)
    _check(k, 3000, 0.2)


def test_zero_noise_is_the_program(orc):
    c = W.plain_small(seed=2)
    nc = noise.with_noise(c, noise.NoiseModel())
    assert nc.n == c.n + 1
    a, _, _ = orc.run_shots(c.ops, c.n, 50, seed=1)
    b, _, _ = orc.run_shots(nc.ops, nc.n, 50, seed=1)
    assert np.array_equal(a, b)


def test_structure_kept_and_scratch_bits_checked():
    c = Circuit(2)
    c.loop(3, lambda: c.x(0))
    c.measure(0, 0)
    c.cond(1, 1, lambda: c.h(1), lambda: c.z(1))
    nc = noise.with_noise(c, noise.NoiseModel(p1=0.1, p_meas=0.1))
    kinds = nc.ops["kind"]
    assert int((kinds == int(Kind.LOOP)).sum()) == 1
    # one channel per gate: the loop body holds x and its channel's decision
    loop = nc.ops[kinds == int(Kind.LOOP)][0]
    assert int(loop["loop_k"]) == 3 and int(loop["body_len"]) > 1
    bad = Circuit(1)
    bad.measure(0, 62)
    with pytest.raises(ValueError):
        noise.with_noise(bad, noise.NoiseModel(p1=0.1))
    with pytest.raises(ValueError):
        noise.NoiseModel(p1=1.5)


def test_noisy_repetition_code_statistics(orc):
    """Distance-3 repetition code, one round, bit flips of probability p on each
    data qubit before the round (as a Pauli channel with px = p), decoded by
    the round's feed-forward: a logical error needs two or more flips, so the
    final data readout (majority after correction) is wrong with probability
    3p^2(1-p) + p^3."""
    p = 0.2
    d = 3
    c = Circuit(2 * d)  # data 0..2, ancillas 3..4, noise ancilla 5
    for q in range(d):
        noise.pauli_channel(c, q, p, 0.0, 0.0, anc=2 * d - 1)
    rep = W.repetition_code(d, 1)
    c._recs += list(rep._recs)  # same qubits: data 0..2, parity ancillas 3, 4
    shots = 3000
    regs, _, _ = orc.run_shots(c.ops, 2 * d, shots, seed=8)
    data = regs & np.uint64(7)
    wrong = int((data == 7).sum())
    assert set(np.unique(data).tolist()) <= {0, 7}
    _check(wrong, shots, 3 * p * p * (1 - p) + p ** 3)
