"""Scheduling rules of the continuous-batching server, on the CPU with a fake backend."""
import threading
import time

import numpy as np
import pytest

from paper_2604_11599_gb300.serve import Req, Server, footprint_bytes


class FakeBackend:
    def __init__(self, free=10 << 30, batch_s=0.02, large_s=0.03):
        self.free = free
        self.batch_s, self.large_s = batch_s, large_s
        self.batches = []
        self.lock = threading.Lock()
        self.live = 0
        self.peak = 0

    def free_bytes(self):
        return self.free

    def _rec(self, r):
        return (np.arange(r.shots, dtype=np.uint64) * 7919 + np.uint64(r.rid)) % np.uint64(1 << 20)

    def run_batch(self, reqs):
        self.batches.append([r.rid for r in reqs])
        time.sleep(self.batch_s)
        return {r.rid: self._rec(r) for r in reqs}

    def run_large(self, r):
        with self.lock:
            self.live += footprint_bytes(r.n, "c64", 18)
            self.peak = max(self.peak, self.live)
        time.sleep(self.large_s)
        with self.lock:
            self.live -= footprint_bytes(r.n, "c64", 18)
        return self._rec(r)


def _reqs(k, n_of=lambda i: 12, gap=0.002, shots=4):
    return [Req(i, i * gap, n_of(i), np.zeros(0), shots) for i in range(k)]


def test_every_request_completes_with_its_own_records():
    be = FakeBackend()
    srv = Server(be, memory_budget=1 << 40)
    reqs = _reqs(40, n_of=lambda i: 12 if i % 3 else 24)
    res, st = srv.serve(reqs)
    srv.close()
    assert [r.rid for r in res] == list(range(40))
    for r in res:
        assert np.array_equal(r.cregs, be._rec(reqs[r.rid]))
    assert st["requests"] == 40 and st["shots"] == 160
    assert st["p99_s"] >= st["p50_s"] > 0


def test_arrivals_during_a_launch_join_the_next_launch():
    be = FakeBackend(batch_s=0.05)
    srv = Server(be, memory_budget=1 << 40)
    res, st = srv.serve(_reqs(30, gap=0.005))
    srv.close()
    assert len(res) == 30
    assert st["batched_launches"] == len(be.batches) < 30
    assert max(len(b) for b in be.batches) > 1
    assert sorted(sum(be.batches, [])) == list(range(30))


def test_launch_shot_cap():
    be = FakeBackend(batch_s=0.03)
    srv = Server(be, memory_budget=1 << 40, max_launch_shots=10)
    res, _ = srv.serve(_reqs(20, gap=0.0, shots=4))
    srv.close()
    assert len(res) == 20
    assert all(len(b) * 4 <= 10 for b in be.batches)


def test_memory_budget_is_never_exceeded():
    be = FakeBackend(large_s=0.05)
    per = footprint_bytes(26, "c64", 18)
    srv = Server(be, memory_budget=3 * per + 10, large_workers=8)
    res, _ = srv.serve(_reqs(12, n_of=lambda i: 26, gap=0.0))
    srv.close()
    assert len(res) == 12
    assert be.peak <= 3 * per


def test_admission_is_first_come_first_served():
    be = FakeBackend(large_s=0.04)
    per = footprint_bytes(27, "c64", 18)
    srv = Server(be, memory_budget=per + 10, large_workers=4)
    res, _ = srv.serve(_reqs(5, n_of=lambda i: 27, gap=0.0))
    srv.close()
    order = sorted(res, key=lambda r: r.admitted)
    assert [r.rid for r in order] == list(range(5))


def test_request_larger_than_budget_is_rejected():
    srv = Server(FakeBackend(), memory_budget=1 << 20)
    with pytest.raises(ValueError, match="more than the whole budget"):
        srv.serve(_reqs(1, n_of=lambda i: 30, gap=0.0))
    srv.close()


def test_large_requests_start_shortest_first():
    """Admitted large requests wait for a worker; the one with the least
    estimated work starts first (arrival order breaks ties)."""
    be = FakeBackend(large_s=0.03)
    started = []
    run = be.run_large

    def spy(r):
        started.append(r.rid)
        return run(r)

    be.run_large = spy
    srv = Server(be, memory_budget=1 << 40, large_workers=1)
    reqs = [Req(0, 0.0, 26, np.zeros(0), 4), Req(1, 0.0, 24, np.zeros(0), 4), Req(2, 0.0, 22, np.zeros(0), 4),
            Req(3, 0.0, 23, np.zeros(0), 4)]
    res, _ = srv.serve(reqs)
    srv.close()
    assert len(res) == 4
    assert started == [2, 3, 1, 0]
    srv = Server(FakeBackend(large_s=0.01), memory_budget=1 << 40, large_workers=1, large_order="fifo")
    be2 = srv.backend
    started.clear()
    run2 = be2.run_large
    be2.run_large = lambda r: (started.append(r.rid), run2(r))[1]
    srv.serve(reqs)
    srv.close()
    assert started == [0, 1, 2, 3]
