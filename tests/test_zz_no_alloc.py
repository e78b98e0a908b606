"""sv_expval_static (no device allocation by the library) agrees with sv_expval
and with the oracle.

sv_expval_static serves callers whose device memory is entirely managed by
their own allocator or pool, or whose loops cannot afford cudaMalloc's
implicit device synchronisation: it keeps its scratch in a static device
array instead of allocating.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W
from paper_2604_11599_gb300.ir import PAULI_DTYPE

pytestmark = pytest.mark.gpu

EXP_TOL = {"c64": 1e-5, "c128": 1e-10}


def _random_paulis(seed, n, count, x_prob=0.7):
    r = np.random.default_rng(seed)
    out = np.zeros(count, dtype=PAULI_DTYPE)
    for t in range(count):
        x = int(r.integers(0, 1 << n)) if r.random() < x_prob else 0
        z = int(r.integers(0, 1 << n))
        out[t] = (x, z, float(r.normal()))
    return out


def _sv():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    return sv


# (n, term set): several X groups; one X group of 40 Z-only terms split over two
# launches that reuse the scratch and its counter; exactly the 64-term limit;
# states small enough for a one-CTA grid (n = 3, 5)
CASES = [
    (13, lambda n: W.heisenberg_fields(seed=3, n=n, n_terms=60)),
    (13, lambda n: _random_paulis(11, n, 37)),
    (13, lambda n: _random_paulis(12, n, 40, x_prob=0.0)),
    (13, lambda n: _random_paulis(13, n, 64)),
    (3, lambda n: _random_paulis(14, n, 20)),
    (5, lambda n: _random_paulis(15, n, 64, x_prob=0.3)),
]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_static_scratch_expval_matches_sv_expval(dtype, orc):
    import torch

    sv = _sv()
    stream = torch.cuda.current_stream().cuda_stream
    for k, (n, make) in enumerate(CASES):
        c = W.random_static(2024 + k, n, 80)
        terms = make(n)
        ref = orc.run(c.ops, n)
        want_orc, _ = orc.expval(ref.psi, terms)
        with sv.State(n, dtype) as st:
            st.run(c.ops)
            state_ptr = st._buf.data_ptr()
            _, want = st.expval(terms)
            for _ in range(2):  # two calls in a row share the static scratch
                out = torch.full((len(terms),), float("nan"), dtype=torch.float64, device="cuda")
                sv.sv_expval_static(state_ptr, n, dtype, terms, out.data_ptr(), stream)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                assert np.isfinite(got).all()
                assert np.max(np.abs(got - want)) <= EXP_TOL[dtype], (n, len(terms))
                assert np.max(np.abs(got - want_orc)) <= EXP_TOL[dtype], (n, len(terms))


def test_static_scratch_rejects_sizes_beyond_its_limit():
    import torch

    sv = _sv()
    with sv.State(8, "c64") as st:
        too_many = _random_paulis(5, 8, 65)
        out = torch.zeros(65, dtype=torch.float64, device="cuda")
        with pytest.raises(sv.SVError, match="at most 64"):
            sv.sv_expval_static(st._buf.data_ptr(), 8, "c64", too_many, out.data_ptr())


def test_static_scratch_rejects_host_pointers():
    import torch

    sv = _sv()
    with sv.State(6, "c64") as st:
        terms = _random_paulis(6, 6, 4)
        host = np.zeros(4, dtype=np.float64)
        with pytest.raises(sv.SVError, match="ARG"):
            sv.sv_expval_static(st._buf.data_ptr(), 6, "c64", terms, host.ctypes.data)
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        with pytest.raises(sv.SVError, match="ARG"):
            sv.sv_expval_static(host.ctypes.data, 6, "c64", terms, out.data_ptr())
