"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import Circuit, Gate

from paritylib import AMP_TOL, EXP_TOL, BAND, compare_run

pytestmark = pytest.mark.gpu

DTYPES = ["c64", "c128"]


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


# --------------------------------------------------------------------------- static circuits
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 11, 12, 13, 15, 17])
def test_static_every_gate(svmod, orc, dtype, n):
    """Random circuits over the whole gate vocabulary incl. dense 1..4-qubit unitaries
    and parameter references, several tiles and register stages."""
    for seed in range(3):
        k = min(n, 1 + (seed + n) % 4)
        c = W.random_static(100 * n + seed, n, 60, dense_k=k, params=5)
        params = np.random.default_rng(seed).uniform(-3, 3, size=5)
        with svmod.State(n, dtype) as st:
            st.set_dense_pool(c.pool)
            compare_run(st, orc, c.ops, n, dtype, params=params, pool=c.pool)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tile,low", [(10, 2), (10, 5), (12, 3), (12, 6), (13, 4), (14, 5)])
def test_tuning_does_not_change_results(svmod, orc, dtype, tile, low):
    n = 16
    c = W.layered(3, n, layers=6)
    with svmod.State(n, dtype) as st:
        st.set_tuning(tile, low, 0)
        compare_run(st, orc, c.ops, n, dtype, seed=1)


@pytest.mark.parametrize("dtype", DTYPES)
def test_max_pass_gates_one_gate_per_pass(svmod, orc, dtype):
    n = 14
    c = W.random_static(7, n, 50, params=0)
    with svmod.State(n, dtype) as st:
        st.set_tuning(0, 0, 1)
        compare_run(st, orc, c.ops, n, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_specialised_kernels_parity(svmod, orc, dtype):
    """Per-program compiled pass kernels (sv_set_jit) give the same records and
    amplitudes as the oracle, for static, dense and dynamic programs."""
    import torch

    cases = [(W.layered(2, 16, layers=6), 16, 0), (W.random_static(21, 14, 80, dense_k=3, params=3), 14, 3),
             (W.random_dynamic(9, 15, n_ops=70, dense_k=2), 15, 0)]
    for c, n, npar in cases:
        params = np.random.default_rng(n).uniform(-2, 2, size=npar) if npar else None
        with svmod.State(n, dtype) as st:
            st.set_jit(True)
            st.set_dense_pool(c.pool)
            for shot in range(3):
                compare_run(st, orc, c.ops, n, dtype, params=params, seed=4, shot=shot, pool=c.pool)
            prog = st.prepare(c.ops)
            dp = None if params is None else torch.tensor(params, device="cuda")
            st.launch(prog, dp, seed=4, shot=0)
            st.sync()
            assert prog.stats["specialised"] == 1


@pytest.mark.parametrize("dtype", DTYPES)
def test_factored_rotations_edge_angles(svmod, orc, dtype):
    """RX / RY / RZ / phase gates run with their scalar factor taken out (form
    chosen by |cos| vs |sin|; the pass applies the product of the factors when it
    stores and scales its measurement table by its squared modulus).  Angles at
    and around the form switch and the zeros of cos and sin, with measurements
    and resets inside the same passes."""
    n = 13
    edge = [0.0, math.pi / 2, math.pi, 3 * math.pi / 2, 2 * math.pi, 3 * math.pi, -math.pi,
            math.pi - 1e-7, math.pi + 1e-7, 1e-7, math.pi / 2 + 1e-9, 7.5]
    rng = np.random.default_rng(17)
    for trial in range(3):
        c = Circuit(n)
        for q in range(n):
            c.h(q)
        for layer in range(4):
            for q in range(n):
                th = float(edge[rng.integers(len(edge))])
                [c.rx, c.ry, c.rz, c.p][int(rng.integers(4))](q, th)
            for q in range(0, n - 1, 2):
                c.cx(q, q + 1)
            c.measure(int(rng.integers(n)), layer)
            c.reset(int(rng.integers(n)))
            c.s(int(rng.integers(n)))
            c.t(int(rng.integers(n)))
        with svmod.State(n, dtype) as st:
            for jit in (False, True):
                st.set_jit(jit)
                for shot in range(3):
                    compare_run(st, orc, c.ops, n, dtype, seed=trial, shot=shot)


@pytest.mark.parametrize("jit", [False, True])
def test_dense4_tensor_cores_parity(svmod, orc, jit):
    """Dense four-qubit unitaries on the tensor cores (complex64, 2^12-amplitude
    tiles): oracle parity, and a result that differs from the FP32-pipe path at
    the rounding level only (so the tensor-core path is the one that ran)."""
    for n in (12, 14, 17):
        c = W.dense_layers(40 + n, n, layers=4)
        with svmod.State(n, "c64") as st:
            st.set_jit(jit)
            st.set_dense_pool(c.pool)
            compare_run(st, orc, c.ops, n, "c64", pool=c.pool)
            a_tc = st.amplitudes()
            st.set_dense_tc(False)
            compare_run(st, orc, c.ops, n, "c64", pool=c.pool)
            a_alu = st.amplitudes()
        assert not np.array_equal(a_tc, a_alu)
        assert float(np.max(np.abs(a_tc - a_alu))) <= AMP_TOL["c64"]


def test_dense4_tensor_cores_in_dynamic_programs(svmod, orc):
    """Dense four-qubit gates beside measurement, reset and feed-forward (the
    collapse is fused into the tile load that feeds the tensor-core stage)."""
    n = 14
    with svmod.State(n, "c64") as st:
        for seed in range(4):
            c = W.random_dynamic(700 + seed, n, n_ops=70, dense_k=4)
            st.set_dense_pool(c.pool)
            for shot in range(3):
                compare_run(st, orc, c.ops, n, "c64", seed=seed, shot=shot, pool=c.pool)


# --------------------------------------------------------------------------- dynamic circuits
@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [2, 4, 6, 9, 13, 16])
def test_random_dynamic_programs(svmod, orc, dtype, n, jit):
    """Measures, resets, nested if/else on 1-3 bit predicates, loops, dense gates
    (generic and per-program specialised kernels)."""
    stats = {}
    with svmod.State(n, dtype) as st:
        st.set_jit(jit)
        for seed in range(6):
            c = W.random_dynamic(1000 * n + seed, n, n_ops=70, dense_k=min(n, 2))
            st.set_dense_pool(c.pool)
            for shot in range(4):
                compare_run(st, orc, c.ops, n, dtype, seed=seed, stream=n, shot=shot, pool=c.pool, stats=stats)
    assert stats["draws"] > 20


def test_plain_small_config_records(svmod, orc):
    """Plain path, complex128, n=5, 1,000 shots of the seeded feed-forward program:
    every record bit-exact (near-threshold draws counted)."""
    c = W.plain_small()
    stats = {}
    with svmod.State(5, "c128") as st:
        for shot in range(1000):
            compare_run(st, orc, c.ops, 5, "c128", seed=0, shot=shot, check_amps=(shot % 50 == 0), stats=stats,
                        label="n=5 c128 feed-forward program, 1,000 shots (plain path)")
    assert stats["draws"] == 5000
    assert stats.get("forced", 0) == 0


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [12, 18, 21])
def test_layered_config_small_sizes(svmod, orc, dtype, n, jit):
    """The layered measure/reset/cond workload at sizes the oracle runs in seconds
    (generic and per-program specialised kernels)."""
    c = W.layered(2, n, layers=20 if n <= 18 else 8)
    with svmod.State(n, dtype) as st:
        st.set_jit(jit)
        for shot in range(2):
            compare_run(st, orc, c.ops, n, dtype, seed=0, shot=shot, label=f"layered n={n} {dtype} (small sizes)")


@pytest.mark.parametrize("dtype", DTYPES)
def test_conditional_reset_always_zero(svmod, dtype):
    """Fig. 2 / Sec. IV-C conditional reset, 10^4 shots: |0> on every shot."""
    for minus in (True, False):
        c = W.conditional_reset(minus)
        with svmod.State(1, dtype) as st:
            ones = 0
            for s in range(0, 10000, 97):
                ones += st.run(c.ops, shot=s) & 1
                a = st.amplitudes()
                assert abs(a[1]) == 0 and abs(abs(a[0]) - 1) < AMP_TOL[dtype]
            cregs, _ = st.sample(c.ops, 10000)
            assert 4700 < int(cregs.sum()) < 5300


@pytest.mark.parametrize("dtype", DTYPES)
def test_teleportation_uncompute(svmod, dtype):
    rng = np.random.default_rng(4)
    with svmod.State(3, dtype) as st:
        seen = set()
        for trial in range(5):
            th, ph, la = rng.uniform(0, 2 * math.pi, size=3)
            c = W.teleport_uncompute(th, ph, la)
            for s in range(16):
                seen.add(st.run(c.ops, shot=s, stream_id=trial))
                a = st.amplitudes().reshape(2, 4)
                assert np.sum(np.abs(a[1]) ** 2) < 10 * AMP_TOL[dtype] ** 2 + 1e-12
        assert seen == {0, 1, 2, 3}


# --------------------------------------------------------------------------- edge cases
@pytest.mark.parametrize("dtype", DTYPES)
def test_edge_programs(svmod, orc, dtype):
    n = 15
    cases = []
    c = Circuit(n)  # empty program
    cases.append(c)
    c = Circuit(n)  # measurement first, then measure the same qubit again
    c.measure(3, 0); c.measure(3, 1); c.reset(3); c.measure(3, 2)
    cases.append(c)
    c = Circuit(n)  # reset with outcome 1 on qubits outside the tile (tile-pair path)
    for q in (14, 13, 12):
        c.x(q)
    c.h(14)
    c.reset(14); c.reset(13); c.reset(12)
    for q in range(5):
        c.h(q)
    c.measure(0, 0)
    cases.append(c)
    c = Circuit(n)  # a measurement group on more than four qubits
    for q in range(n):
        c.h(q)
    for q in range(7):
        c.measure(q, q)
    c.cond(0b11, 0b01, lambda: c.x(9), lambda: c.z(9))
    cases.append(c)
    c = Circuit(n)  # predicate decided inside the same measurement group
    c.h(0); c.h(1)
    c.measure(0, 0)
    c.cond(1, 1, lambda: c.measure(1, 1), lambda: c.reset(1))
    c.h(2)
    cases.append(c)
    c = Circuit(n)  # loop(0), loop with only control flow, cond with empty then
    c.loop(0, lambda: c.x(0))
    c.h(5)
    c.measure(5, 5)
    c.cond(1 << 5, 1 << 5, lambda: None, lambda: c.x(6))
    c.loop(3, lambda: c.cond(1 << 5, 0, lambda: (c.h(5), c.measure(5, 5))))
    cases.append(c)
    c = Circuit(n)  # program ending in a reset (final projector flush)
    c.h(10); c.cx(10, 2); c.reset(10)
    cases.append(c)
    with svmod.State(n, dtype) as st:
        for c in cases:
            for shot in range(5):
                compare_run(st, orc, c.ops, n, dtype, seed=3, shot=shot)


@pytest.mark.parametrize("dtype", DTYPES)
def test_errors_are_status_codes(svmod, dtype):
    with svmod.State(4, dtype) as st:
        c = Circuit(5)
        c.x(4)
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            st.run(c.ops)
        c = Circuit(4)
        c.rx(0, __import__("paper_2604_11599_gb300.ir", fromlist=["Param"]).Param(3))
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            st.run(c.ops, params=[0.1])
        c = Circuit(4)
        c.measure(0, 64)
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            st.run(c.ops)
        ops = Circuit(4).cond(1, 1, lambda: None).ops
        ops["then_len"] = 5
        with pytest.raises(svmod.SVError, match="SV_ERR_ARG"):
            st.run(ops)
        # the handle stays usable after errors
        c = Circuit(4)
        c.x(1)
        assert st.run(c.ops) == 0
        assert abs(st.amplitudes()[2]) == pytest.approx(1.0)
    with pytest.raises(svmod.SVError):
        svmod.State(40, dtype)


# --------------------------------------------------------------------------- sampling and expval
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [3, 10, 14])
def test_terminal_samples_vs_oracle(svmod, orc, dtype, n):
    c = W.random_static(55 + n, n, 40)
    with svmod.State(n, dtype) as st:
        st.run(c.ops)
        got = st.sample_state(2000, seed=4, stream_id=1)
    ref = orc.run(c.ops, n)
    want, margin = orc.sample(ref.psi, 2000, seed=4, stream=1)
    band = 1e-12 if dtype == "c128" else 1e-4
    bad = (got != want) & (margin > band)
    assert not bad.any(), f"{int(bad.sum())} samples differ away from CDF ties"
    assert (got == want).mean() > 0.99


@pytest.mark.parametrize("dtype", DTYPES)
def test_terminal_samples_large_state_vs_oracle(svmod, orc, dtype):
    """A state of many CDF blocks (n=19: 64 blocks of 256 runs) against the oracle."""
    n = 19
    c = W.layered(31, n, layers=3)
    with svmod.State(n, dtype) as st:
        st.run(c.ops, seed=2)
        got = st.sample_state(4000, seed=5, stream_id=3)
    ref = orc.run(c.ops, n, seed=2)
    want, margin = orc.sample(ref.psi, 4000, seed=5, stream=3)
    band = 1e-12 if dtype == "c128" else 1e-4
    bad = (got != want) & (margin > band)
    assert not bad.any(), f"{int(bad.sum())} samples differ away from CDF ties"


@pytest.mark.parametrize("dtype", DTYPES)
def test_terminal_samples_sparse_and_uniform_states(svmod, orc, dtype):
    """Closed forms: a basis state |x> always gives x; GHZ gives 0 or 2^n - 1
    only (runs and blocks of zeros between them); |+>^n gives floor(u 2^n)
    (all |amp|^2 equal, so the CDF is proportional to i + 1 up to the
    summation's rounding; draws within 1e-6 of an index boundary are left
    out)."""
    import torch

    n = 20
    for x in (0, 1, 12345, (1 << n) - 1, 1 << 19):
        c = Circuit(n)
        for q in range(n):
            if (x >> q) & 1:
                c.x(q)
        with svmod.State(n, dtype) as st:
            st.run(c.ops)
            assert (st.sample_state(500, seed=x) == x).all()
            dev = torch.empty(300, dtype=torch.int64, device="cuda")
            st.sample_state_device(dev, seed=x)
            assert (dev.cpu().numpy() == x).all()
    with svmod.State(n, dtype) as st:
        st.run(W.ghz(n).ops)
        got = st.sample_state(4000, seed=7)
        assert set(np.unique(got).tolist()) == {0, (1 << n) - 1}
        assert 1800 < int((got == 0).sum()) < 2200
        c = Circuit(n)
        for q in range(n):
            c.h(q)
        st.run(c.ops)
        got = st.sample_state(3000, seed=8, stream_id=2, shot0=11)
    t = np.array([orc.uniform(8, 2, 11 + s, 1 << 32) * (1 << n) for s in range(3000)])
    want = np.floor(t).astype(np.uint64)
    frac = t - np.floor(t)
    ok = np.minimum(frac, 1 - frac) > 1e-6
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], want[ok])


@pytest.mark.parametrize("dtype", DTYPES)
def test_sample_program_shots(svmod, orc, dtype):
    c = W.plain_small(seed=3)
    with svmod.State(5, dtype) as st:
        cregs, bits = st.sample(c.ops, 200, seed=2, terminal=True)
    rc, rb, margins = orc.run_shots(c.ops, 5, 200, seed=2, terminal=True)
    ok = margins > BAND[dtype]
    assert (cregs[ok] == rc[ok]).all()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [4, 11, 16])
def test_expval_vs_oracle(svmod, orc, dtype, n):
    c = W.random_static(77 + n, n, 60)
    terms = W.heisenberg_fields(seed=9, n=n, n_terms=10 * n)
    with svmod.State(n, dtype) as st:
        st.run(c.ops)
        tot, per = st.expval(terms)
    ref = orc.run(c.ops, n)
    rper, rtot = orc.expval(ref.psi, terms)
    assert np.max(np.abs(per - rper)) <= EXP_TOL[dtype]
    assert abs(tot - rtot) <= EXP_TOL[dtype] * max(1.0, float(np.abs(terms["coeff"]).sum()))


def test_state_tensor_view_is_zero_copy(svmod):
    import torch

    with svmod.State(6, "c64") as st:
        c = Circuit(6)
        c.x(2)
        st.run(c.ops)
        t = st.tensor()
        assert t.is_cuda and t.dtype == torch.complex64
        assert abs(complex(t[4].item()) - 1) < 1e-7


def test_program_outliving_its_state(svmod):
    """A prepared program freed after its state was closed: the free touches
    nothing of the state, and a launch of such a program on a new state is an
    argument error (not a launch of another state's plan)."""
    c = W.layered(5, 12, layers=2)
    st = svmod.State(12, "c64")
    prog = st.prepare(c.ops)
    st.launch(prog)
    st.close()
    st2 = svmod.State(12, "c64")
    with pytest.raises(svmod.SVError):
        st2.launch(prog)
    prog.free()
    prog2 = st2.prepare(c.ops)
    st2.launch(prog2)
    del prog2  # freed while its state is alive
    st2.close()
