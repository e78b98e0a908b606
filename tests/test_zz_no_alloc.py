"""sv_expval_static (no device allocation by the library) agrees with sv_expval.

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


def _random_paulis(seed, n, count):
    r = np.random.default_rng(seed)
    out = np.zeros(count, dtype=PAULI_DTYPE)
    for t in range(count):
        x = int(r.integers(0, 1 << n)) if r.random() < 0.7 else 0
        z = int(r.integers(0, 1 << n))
        out[t] = (x, z, float(r.normal()))
    return out


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_static_scratch_expval_matches_sv_expval(dtype):
    import torch

    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    n = 13
    c = W.random_static(2024, n, 80)
    stream = torch.cuda.current_stream().cuda_stream
    with sv.State(n, dtype) as st:
        st.run(c.ops)
        state_ptr = st._buf.data_ptr()
        first = W.heisenberg_fields(seed=3, n=n, n_terms=60)
        second = _random_paulis(11, n, 37)
        for terms in (first, second):  # two calls in a row share the static scratch
            _, want = st.expval(terms)
            out = torch.full((len(terms),), float("nan"), dtype=torch.float64, device="cuda")
            sv.sv_expval_static(state_ptr, n, dtype, terms, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.max(np.abs(got - want)) <= EXP_TOL[dtype]


def test_static_scratch_rejects_sizes_beyond_its_limit():
    import torch

    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import sv

    with sv.State(8, "c64") as st:
        too_many = _random_paulis(5, 8, 65)
        out = torch.zeros(65, dtype=torch.float64, device="cuda")
        with pytest.raises(sv.SVError, match="at most 64"):
            sv.sv_expval_static(st._buf.data_ptr(), 8, "c64", too_many, out.data_ptr())
