"""Serving: each request's records are the same alone and in the mix (and on the plain path)."""
import numpy as np
import pytest

from paper_2604_11599_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_alone_vs_mix_and_plain_path():
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import serve

    stream = W.serving_stream(seed=10, gen_seed=11, rate=400.0, duration=1.0, n_lo=10, n_hi=24,
                              d_lo=4, d_hi=16, max_shots=48, limit=64)
    reqs = serve.requests_from_stream(stream)
    assert any(r.n > 21 for r in reqs) and any(r.n <= 21 for r in reqs)
    be = serve.GpuBackend("c64", seed=5)
    srv = serve.Server(be, batch_max_n=21, large_workers=3)
    mix, stats = srv.serve(reqs)
    assert stats["requests"] == len(reqs)
    for q in reqs[:12]:
        q0 = serve.Req(q.rid, 0.0, q.n, q.ops, q.shots)
        alone, _ = srv.serve([q0])
        assert np.array_equal(alone[0].cregs, mix[q.rid].cregs), q.rid
    for q in reqs[:6]:  # branched large path and one trajectory per shot give the same records
        assert np.array_equal(be.run_large(q), mix[q.rid].cregs), q.rid
        assert np.array_equal(be.run_plain(q), mix[q.rid].cregs), q.rid
    srv.close()
    # the per-shot engines (branching off) agree as well
    be2 = serve.GpuBackend("c64", seed=5, branching=False)
    srv2 = serve.Server(be2, batch_max_n=21, large_workers=3)
    mix2, _ = srv2.serve(reqs[:24])
    for q in reqs[:24]:
        assert np.array_equal(mix2[q.rid].cregs, mix[q.rid].cregs), q.rid
    srv2.close()


def test_alone_vs_mix_64_requests_with_large_states():
    """64 seeded requests of 10-27 qubits (eight of 25 or more, on resident
    states), served together with continuous batching and then each alone:
    every record is the same (the draws of shot s of request r are keyed by
    (seed, r, s, draw index), and the engines are deterministic)."""
    from paper_2604_11599_gb300 import build

    build.build()
    from paper_2604_11599_gb300 import serve

    stream = W.serving_stream(seed=20, gen_seed=120, rate=200.0, duration=1.0, n_lo=10, n_hi=27, d_lo=10,
                              d_hi=30, max_shots=128, limit=64)
    reqs = serve.requests_from_stream(stream)
    assert len(reqs) == 64 and sum(r.n >= 25 for r in reqs) >= 5
    be = serve.GpuBackend("c64", seed=9)
    srv = serve.Server(be, batch_max_n=18, large_workers=4)
    mix, stats = srv.serve(reqs)
    assert stats["requests"] == 64
    paths = {r.rid: r.path for r in mix}
    assert "large" in paths.values() and "batch" in paths.values()
    for q in reqs:
        alone, _ = srv.serve([serve.Req(q.rid, 0.0, q.n, q.ops, q.shots)])
        assert np.array_equal(alone[0].cregs, mix[q.rid].cregs), (q.rid, q.n)
    srv.close()
