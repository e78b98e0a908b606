"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: numpy's independent Philox,
scipy matrix exponentials, dense Kronecker products, closed forms of the
paper's own validation circuits (Sec. IV-A.2, Fig. 2, Sec. IV-C, Sec. IV-D),
a stabilizer tableau, or a statistical law.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import GATE_ARITY, Circuit, Gate, pauli_terms

import refsim as R

RNG = np.random.default_rng(1234)


# --------------------------------------------------------------------------- Philox
def test_philox_matches_numpy(orc):
    for _ in range(50):
        ctr = [int(v) for v in RNG.integers(0, 2**63, size=4, dtype=np.int64)]
        ctr[0] |= int(RNG.integers(0, 2)) << 63
        key = [int(v) for v in RNG.integers(0, 2**63, size=2, dtype=np.int64)]
        assert list(orc.philox(ctr, key)) == list(R.np_philox_block(ctr, key))
    # counter words 1..3 and both key words all matter
    assert list(orc.philox([0, 1, 0, 0], [0, 0])) == list(R.np_philox_block([0, 1, 0, 0], [0, 0]))
    assert list(orc.philox([0, 0, 0, 5], [0, 7])) == list(R.np_philox_block([0, 0, 0, 5], [0, 7]))


def test_uniform_key_and_counter_mapping(orc):
    for seed, stream, shot, m in [(0, 0, 0, 0), (1, 2, 3, 4), (2**40, 17, 999, 2**32), (5, 0, 1, 1)]:
        assert orc.uniform(seed, stream, shot, m) == R.np_uniform(seed, stream, shot, m)


# --------------------------------------------------------------------------- gate matrices
@pytest.mark.parametrize("g", list(Gate))
def test_gate_matrices_vs_generators(orc, g):
    ang = list(RNG.uniform(-2 * math.pi, 2 * math.pi, size=3))
    shape, m = orc.gate_matrix(int(g), ang)
    kind, ref = R.ref_gate(g.name, ang)
    assert shape == {"1q": 1, "ctrl": 2, "swap": 3}[kind]
    if kind != "swap":
        np.testing.assert_allclose(m, ref, atol=1e-14)
        np.testing.assert_allclose(m.conj().T @ m, np.eye(2), atol=1e-14)


# --------------------------------------------------------------------------- gate application
@pytest.mark.parametrize("seed", range(8))
def test_static_circuits_vs_dense_kronecker(orc, seed):
    n = 2 + seed % 4
    c = W.random_static(seed, n, 40, dense_k=min(3, n) if seed % 2 else 0, params=4)
    params = RNG.uniform(-3, 3, size=4)
    tr = orc.run(c.ops, n, params, pool=c.pool)
    assert tr.status == 0
    ref = R.static_state(c.ops, n, params, c.pool)
    np.testing.assert_allclose(tr.psi, ref, atol=1e-13)


def test_every_gate_on_every_qubit_pair(orc):
    n = 3
    for g in Gate:
        nq, na = GATE_ARITY[g]
        pairs = [(a,) for a in range(n)] if nq == 1 else [(a, b) for a in range(n) for b in range(n) if a != b]
        for qs in pairs:
            c = Circuit(n)
            for q in range(n):  # a generic input state
                c.u(q, 0.3 + q, 0.7 * q, 1.1 - q)
            c.gate(g, list(qs), list(RNG.uniform(0, 6, size=na)))
            tr = orc.run(c.ops, n)
            np.testing.assert_allclose(tr.psi, R.static_state(c.ops, n), atol=1e-13)


def test_dense_gate_bit_order(orc):
    n = 4
    r = np.random.default_rng(5)
    for k in (1, 2, 3, 4):
        qs = [int(v) for v in r.permutation(n)[:k]]
        a = r.normal(size=(1 << k, 1 << k)) + 1j * r.normal(size=(1 << k, 1 << k))
        u, _ = np.linalg.qr(a)
        c = Circuit(n)
        for q in range(n):
            c.u(q, 0.2 + q, 0.5, 0.9 * q)
        c.dense(qs, u)
        tr = orc.run(c.ops, n, pool=c.pool)
        np.testing.assert_allclose(tr.psi, R.static_state(c.ops, n, pool=c.pool), atol=1e-13)


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 7])
def test_ghz_amplitudes(orc, n):
    tr = orc.run(W.ghz(n).ops, n)
    ref = np.zeros(1 << n, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(tr.psi, ref, atol=1e-15)


@pytest.mark.parametrize("n,x", [(3, 5), (4, 11), (6, 37)])
def test_qft_closed_form(orc, n, x):
    """QFT|x> = sum_k e^{2 pi i x k / 2^n} |k> / sqrt(2^n) (Sec. IV-A.2 lists QFT)."""
    tr = orc.run(W.qft_on_basis(n, x).ops, n)
    k = np.arange(1 << n)
    ref = np.exp(2j * math.pi * x * k / (1 << n)) / math.sqrt(1 << n)
    np.testing.assert_allclose(tr.psi, ref, atol=1e-13)


@pytest.mark.parametrize("n,secret", [(4, 0b1011), (6, 0b100110), (5, 0)])
def test_bernstein_vazirani(orc, n, secret):
    """Sec. IV-A.2 lists Bernstein-Vazirani: the measured inputs equal the secret on every shot."""
    c = W.bernstein_vazirani(n, secret)
    cregs, _, _ = orc.run_shots(c.ops, n + 1, 32)
    assert set(int(v) for v in cregs) == {secret}


@pytest.mark.parametrize("minus", [True, False])
def test_conditional_reset_always_zero(orc, minus):
    """Fig. 2 / Sec. IV-C: measure |+> or |->, X if 1: the state is exactly |0> on every shot
    (stronger than the paper's P > 0.999 over 10^4 shots), and the outcomes are fair coin flips."""
    c = W.conditional_reset(minus)
    ones = 0
    shots = 10000
    for s in range(shots):
        tr = orc.run(c.ops, 1, shot=s)
        assert tr.psi[1] == 0 and abs(abs(tr.psi[0]) - 1) < 1e-15
        ones += tr.creg & 1
    assert stats.binomtest(int(ones), shots, 0.5).pvalue > 1e-4


def test_teleportation_returns_to_zero(orc):
    """Sec. IV-A.2: teleport U|0>, uncompute on the receiver, which returns to |0>
    deterministically; all four measurement records occur."""
    r = np.random.default_rng(3)
    seen = set()
    for trial in range(6):
        th, ph, la = r.uniform(0, 2 * math.pi, size=3)
        c = W.teleport_uncompute(th, ph, la)
        for s in range(40):
            tr = orc.run(c.ops, 3, shot=s, stream=trial)
            psi = tr.psi.reshape(2, 4)  # [q2][q1 q0]
            assert np.sum(np.abs(psi[1]) ** 2) < 1e-28
            assert abs(np.sum(np.abs(psi[0]) ** 2) - 1) < 1e-14
            seen.add(tr.creg)
    assert seen == {0, 1, 2, 3}


def test_hea_zz_closed_form_and_gradient(orc):
    """Sec. IV-A.2 / IV-D VQE check, H = Z0 Z1 on a one-layer two-qubit HEA:
    CX(0,1) maps Z0Z1 to Z1, so <H> = cos(theta_RY on q1) and only that
    parameter has a gradient, -sin(theta)."""
    c = W.hea(n=2, layers=1)
    terms = pauli_terms([("Z0 Z1", 1.0)])
    for _ in range(10):
        p = RNG.uniform(-math.pi, math.pi, size=4)
        e = orc.energy(c.ops, 2, p, terms)
        assert abs(e - math.cos(p[1])) < 1e-14
        g = orc.param_shift_grad(c.ops, 2, p, terms)
        np.testing.assert_allclose(g, [0, -math.sin(p[1]), 0, 0], atol=1e-14)


# --------------------------------------------------------------------------- measurement rule
def test_measure_record_bit_exact_vs_numpy_draws(orc):
    """RY(theta) then measure: p0 = cos^2(theta/2); outcome = (u >= p0) with u
    from numpy's Philox at key (seed, stream), counter (shot, m)."""
    for shot in range(200):
        th = 0.3 + 0.01 * shot
        c = Circuit(1)
        c.ry(0, th)
        c.measure(0, 0)
        tr = orc.run(c.ops, 1, seed=9, stream=4, shot=shot)
        u = R.np_uniform(9, 4, shot, 0)
        p0 = math.cos(th / 2) ** 2
        if abs(u - p0) > 1e-12:
            assert tr.creg == int(u >= p0)


def test_draw_index_counts_resets_loops_and_branches(orc):
    """m counts every executed measure and reset, including loop iterations and
    taken branches; skipped branches draw nothing."""
    c = Circuit(3)
    c.h(0)
    c.reset(0)              # m = 0
    c.h(1)
    c.measure(1, 0)         # m = 1
    c.cond(1, 1, lambda: (c.h(2), c.measure(2, 1)), lambda: (c.h(2), c.measure(2, 2)))  # m = 2
    c.loop(3, lambda: (c.h(0), c.measure(0, 3)))  # m = 3, 4, 5
    for shot in range(64):
        tr = orc.run(c.ops, 3, seed=1, stream=2, shot=shot)
        u = [R.np_uniform(1, 2, shot, m) for m in range(6)]
        b0 = int(u[1] >= 0.5)
        want = b0 | (int(u[2] >= 0.5) << (1 if b0 else 2)) | (int(u[5] >= 0.5) << 3)
        assert tr.creg == want
        assert len(tr.draws) == 6


def test_measurement_statistics_chi2(orc):
    """Outcome frequencies of a 3-qubit entangled state follow the Born rule."""
    c = Circuit(3)
    c.ry(0, 1.1); c.cx(0, 1); c.ry(2, 2.3); c.cry(1, 2, 0.7)
    c.measure(0, 0); c.measure(1, 1); c.measure(2, 2)
    probs = np.abs(orc.run(c.ops[:4], 3).psi) ** 2
    shots = 4000
    cregs, _, _ = orc.run_shots(c.ops, 3, shots, seed=11)
    counts = np.bincount(cregs.astype(np.int64), minlength=8)
    mask = probs > 1e-12
    assert counts[~mask].sum() == 0
    assert stats.chisquare(counts[mask], probs[mask] * shots).pvalue > 1e-4


def test_repeat_until_success_probability(orc):
    """loop(4){ if (c==0) { reset; ry(theta); measure } } succeeds with
    probability 1 - cos^8(theta/2) (a binomial law)."""
    th = 1.0
    c = Circuit(1)
    c.loop(4, lambda: c.cond(1, 0, lambda: (c.reset(0), c.ry(0, th), c.measure(0, 0))))
    shots = 4000
    cregs, _, _ = orc.run_shots(c.ops, 1, shots, seed=3)
    p = 1 - math.cos(th / 2) ** 8
    assert stats.binomtest(int(cregs.sum()), shots, p).pvalue > 1e-4


def test_loop_count_and_nested_cond(orc):
    for k in range(0, 6):
        c = Circuit(2)
        c.loop(k, lambda: c.x(0))
        c.measure(0, 0)
        c.cond(1, 1, lambda: c.loop(2, lambda: c.x(1)), lambda: c.x(1))
        tr = orc.run(c.ops, 2)
        assert tr.creg == k % 2
        assert abs(tr.psi[(k % 2) | ((0 if k % 2 else 1) << 1)]) == pytest.approx(1.0)


@pytest.mark.parametrize("seed", range(6))
def test_norm_is_one_after_every_op(orc, seed):
    c = W.random_dynamic(seed, 5, n_ops=80, dense_k=2)
    tr = orc.run(c.ops, 5, pool=c.pool, trace_norms=True, seed=seed)
    assert tr.status == 0 and len(tr.norms) > 10
    np.testing.assert_allclose(tr.norms, 1.0, atol=1e-14)


def test_forced_outcomes_follow_the_given_record(orc):
    c = Circuit(2)
    c.h(0); c.h(1); c.measure(0, 0); c.measure(1, 1)
    for f in ([0, 0], [0, 1], [1, 0], [1, 1]):
        tr = orc.run(c.ops, 2, forced=np.array(f))
        assert tr.creg == f[0] | (f[1] << 1)
        assert abs(tr.psi[f[0] | (f[1] << 1)]) == pytest.approx(1.0)


def test_thread_count_does_not_change_results(orc):
    c = W.layered(2, 14, layers=4)
    old = orc.get_threads()
    orc.set_threads(1)
    a = orc.run(c.ops, 14, seed=0)
    orc.set_threads(4)
    b = orc.run(c.ops, 14, seed=0)
    orc.set_threads(old)
    assert a.creg == b.creg
    assert np.array_equal(a.psi, b.psi)
    assert np.array_equal(a.draws, b.draws)


# --------------------------------------------------------------------------- stabilizer pin
@pytest.mark.parametrize("seed", range(10))
def test_random_clifford_vs_stabilizer_tableau(orc, seed):
    """Sec. IV-A.2 / IV-B static suite (random Cliffords, n in [2,20]): the oracle's
    state is a +1 eigenvector of every stabilizer generator the tableau tracks."""
    n = 2 + seed
    depth = 10 + 9 * seed
    c = W.random_clifford(seed, n, depth)
    tr = orc.run(c.ops, n)
    tab = R.Tableau(n)
    names = {int(g): g.name for g in Gate}
    for op in c.ops:
        nm = names[int(op["gate"])]
        tab.apply(nm, [int(v) for v in op["q"][: (2 if nm in ("CX", "CZ", "SWAP") else 1)]])
    for sign, xm, zm in tab.generators():
        terms = np.zeros(1, dtype=[("x_mask", "<u8"), ("z_mask", "<u8"), ("coeff", "<f8")])
        terms[0] = (xm, zm, 1.0)
        per, _ = orc.expval(tr.psi, terms)
        assert per[0] == pytest.approx(sign, abs=1e-12)


# --------------------------------------------------------------------------- sampling and expval
def test_terminal_sampling_exact_on_uniform_state(orc):
    """|+>^n has CDF c_i = (i+1)/2^n exactly, so the sample is floor(u * 2^n)."""
    n = 6
    c = Circuit(n)
    for q in range(n):
        c.h(q)
    psi = orc.run(c.ops, n).psi
    out, _ = orc.sample(psi, 300, seed=5, stream=1)
    for s in range(300):
        u = R.np_uniform(5, 1, s, 1 << 32)
        assert int(out[s]) == math.floor(u * (1 << n))


def test_terminal_sampling_chi2(orc):
    n = 4
    c = W.random_static(7, n, 30)
    psi = orc.run(c.ops, n).psi
    shots = 20000
    out, _ = orc.sample(psi, shots, seed=2)
    counts = np.bincount(out.astype(np.int64), minlength=1 << n)
    p = np.abs(psi) ** 2
    assert stats.chisquare(counts, p / p.sum() * shots).pvalue > 1e-4


@pytest.mark.parametrize("n", [3, 5])
def test_expval_vs_dense_hamiltonian(orc, n):
    c = W.random_static(11 + n, n, 40)
    psi = orc.run(c.ops, n).psi
    terms = W.heisenberg_fields(seed=9, n=n, n_terms=4 * n)
    per, tot = orc.expval(psi, terms)
    H = R.hamiltonian(n, terms)
    assert tot == pytest.approx(float(np.real(psi.conj() @ H @ psi)), abs=1e-12)
    for t in range(len(terms)):
        P = R.pauli_matrix(n, int(terms[t]["x_mask"]), int(terms[t]["z_mask"]))
        assert per[t] == pytest.approx(float(np.real(psi.conj() @ P @ psi)), abs=1e-13)


def test_gradient_param_shift_vs_finite_differences(orc):
    n = 4
    c = W.hea(n=n, layers=2)
    terms = W.heisenberg_fields(seed=9, n=n, n_terms=20)
    p = np.random.default_rng(8).uniform(-math.pi, math.pi, size=4 * n)
    gs = orc.param_shift_grad(c.ops, n, p, terms)
    gf = orc.finite_diff_grad(c.ops, n, p, terms)
    np.testing.assert_allclose(gs, gf, atol=1e-8)


# --------------------------------------------------------------------------- workload pins
def test_workload_shapes():
    c1 = W.plain_small()
    kinds = np.bincount(c1.ops["kind"], minlength=7)
    assert kinds[3] == 5 and kinds[5] == 10  # 5 measures, 5 cond-resets + 5 if-else
    c2 = W.layered(2, 30)
    g = c2.ops[c2.ops["kind"] == 1]
    assert len(g) == 20 * (30 + 15) + 2 * 5  # + the X (then) and Z (else) gate of each cond
    hea = W.hea()
    assert hea.n_params == 320
    assert len(W.heisenberg_fields()) == 200


def test_sequential_feedforward_rus_pin(orc):
    """Batching circuit with n=4 data qubits: the ancilla's RUS loop succeeds
    within 4 attempts with probability 1 - cos^8(theta_r/2)."""
    c = W.sequential_feedforward(44, 4)
    shots = 3000
    cregs, _, _ = orc.run_shots(c.ops, 5, shots, seed=0)
    ok = int(((cregs >> np.uint64(63)) & np.uint64(1)).sum())
    p = 1 - math.cos(c.rus_theta / 2) ** 8
    assert stats.binomtest(ok, shots, p).pvalue > 1e-4
