"""Noisy programs (channels lowered into the IR) on the GPU engines: records
equal the oracle's away from the near-threshold band, and shot branching and
the batched launch agree with the plain path."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import noise, workloads as W

from paritylib import BAND

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svmod():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


def test_noisy_program_engines_vs_oracle(svmod, orc):
    c = noise.with_noise(W.plain_small(seed=5), noise.NoiseModel(p1=0.02, p2=0.05, p_meas=0.03, p_reset=0.02))
    n, shots = c.n, 200
    want, _, margins = orc.run_shots(c.ops, n, shots, seed=2)
    ok = margins > BAND["c128"]
    assert ok.mean() > 0.95
    with svmod.State(n, "c128") as st:
        plain, _ = st.sample(c.ops, shots, seed=2)
        branched, stats = st.sample_branched(c.ops, shots, seed=2)
    assert np.array_equal(plain[ok], want[ok])
    assert np.array_equal(branched, plain)
    with svmod.Batch("c128") as b:
        p = b.add_program(c.ops, n)
        per_shot = b.run(np.full(shots, p), np.zeros(shots), np.arange(shots), seed=2)
        br, _ = b.sample_branched([p], [0], [shots], seed=2)
    assert np.array_equal(per_shot[ok], want[ok])
    assert np.array_equal(br, per_shot)
    assert 1 <= stats["paths"] <= shots
