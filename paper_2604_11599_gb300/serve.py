"""Continuous-batching request server for dynamic-circuit shots.

Requests (a circuit, its qubit count, a shot count) arrive over time.  The
scheduler admits them first-come first-served while their device-memory
footprint fits the budget, and runs two kinds of work concurrently on the GPU:

* small requests (n <= ``batch_max_n``) join the next persistent batched launch
  (``sv_batch``): every launch takes all shots of all admitted small requests
  that are waiting, so requests that arrive while a launch runs are picked up
  by the next one (continuous batching);
* large requests get a resident state vector and their own CUDA stream in a
  worker pool; their shots run back to back on that stream, overlapping with
  the batched launches and with each other.  Admitted large requests start
  shortest first (estimated work: 2^n x program length x the shots that can
  take distinct outcome paths, capped at 64), so a long request does not hold
  up the short ones behind it; the batched launches run on a high-priority
  stream, so the GPU turns to them between the large requests' kernels.

Shot s of request r uses Philox key (seed, stream = r.rid) and counter
(shot = s, draw index): its record does not depend on what else is running,
so each result is the same alone and in the mix.

The scheduling logic is independent of the GPU: a backend object executes
work, so the admission and batching rules are tested on the CPU with a fake
backend.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


@dataclass
class Req:
    rid: int
    arrival: float      # seconds after the start of the stream
    n: int
    ops: np.ndarray
    shots: int


@dataclass
class Result:
    rid: int
    cregs: np.ndarray
    arrival: float
    admitted: float
    finished: float
    path: str

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint_bytes(n: int, dtype: str, batch_max_n: int = 18) -> int:
    """Device memory a request holds while it runs: its own state vector on
    the large-request path, none beyond the batched engine's fixed slots on
    the small-request path."""
    if n <= batch_max_n:
        return 0
    amp = 8 if dtype == "c64" else 16
    return (1 << max(n, 10)) * amp + (1 << 20)


class GpuBackend:
    """Executes work on the GPU through the C-ABI binding.

    With ``branching`` (default) the shots of a request run by shot
    branching: one trajectory per distinct outcome path, every record equal
    to the one the shot's own trajectory gives on the same engine."""

    def __init__(self, dtype: str = "c64", seed: int = 0, branching: bool = True):
        import torch

        from . import sv

        self.sv, self.torch = sv, torch
        self.dtype, self.seed, self.branching = dtype, seed, branching
        self.batch_stream = torch.cuda.Stream(priority=-1)  # the GPU takes these launches first
        with torch.cuda.stream(self.batch_stream):
            self.batch = sv.Batch(dtype, stream=self.batch_stream.cuda_stream)
        self.prog_ids: dict[int, int] = {}

    def free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info()
        return int(free)

    def run_batch(self, reqs: list[Req]) -> dict[int, np.ndarray]:
        """All shots of these small requests in one persistent launch (one
        launch per walk round with branching)."""
        progs, streams, shots = [], [], []
        for r in reqs:
            if r.rid not in self.prog_ids:
                self.prog_ids[r.rid] = self.batch.add_program(r.ops, r.n)
        if self.branching:
            out, _ = self.batch.sample_branched([self.prog_ids[r.rid] for r in reqs], [r.rid for r in reqs],
                                                [r.shots for r in reqs], seed=self.seed)
            res, k = {}, 0
            for r in reqs:
                res[r.rid] = out[k: k + r.shots]
                k += r.shots
            return res
        for r in reqs:
            progs.append(np.full(r.shots, self.prog_ids[r.rid], dtype=np.uint32))
            streams.append(np.full(r.shots, r.rid, dtype=np.uint64))
            shots.append(np.arange(r.shots, dtype=np.uint64))
        out = self.batch.run(np.concatenate(progs), np.concatenate(streams), np.concatenate(shots), seed=self.seed)
        res, k = {}, 0
        for r in reqs:
            res[r.rid] = out[k: k + r.shots]
            k += r.shots
        return res

    def run_large(self, r: Req) -> np.ndarray:
        """All shots of one request on its own resident state and stream."""
        s = self.torch.cuda.Stream()
        with self.torch.cuda.stream(s):
            with self.sv.State(r.n, self.dtype, stream=s.cuda_stream) as st:
                if self.branching:
                    cregs, _ = st.sample_branched(r.ops, r.shots, seed=self.seed, stream_id=r.rid)
                else:
                    cregs, _ = st.sample(r.ops, r.shots, seed=self.seed, stream_id=r.rid)
        return cregs

    def run_plain(self, r: Req) -> np.ndarray:
        """The plain path: one trajectory per shot on one resident state."""
        with self.sv.State(r.n, self.dtype) as st:
            cregs, _ = st.sample(r.ops, r.shots, seed=self.seed, stream_id=r.rid)
        return cregs


def work_estimate(r: Req) -> float:
    """Relative cost of a request on the large-request path: one trajectory
    sweeps 2^n amplitudes about once per few records, and shot branching runs
    one trajectory per distinct outcome path (at most the shots)."""
    return float(1 << max(r.n, 10)) * max(1, len(r.ops)) * min(max(r.shots, 1), 64)


class Server:
    def __init__(self, backend, dtype: str = "c64", batch_max_n: int = 18, memory_budget: Optional[int] = None,
                 large_workers: int = 4, max_launch_shots: int = 8192, large_order: str = "shortest",
                 clock: Callable[[], float] = time.perf_counter):
        if large_order not in ("shortest", "fifo"):
            raise ValueError("large_order is 'shortest' or 'fifo'")
        self.backend = backend
        self.dtype = dtype
        self.batch_max_n = batch_max_n
        self.max_launch_shots = max_launch_shots
        self.large_order = large_order
        self.large_workers = large_workers
        self.budget = memory_budget if memory_budget is not None else int(0.8 * backend.free_bytes())
        self.pool = ThreadPoolExecutor(max_workers=large_workers)
        self.clock = clock
        self.lock = threading.Lock()

    def serve(self, requests: list[Req], realtime: bool = True, idle_sleep: float = 2e-4) -> tuple[list[Result], dict]:
        """Runs the request stream to completion; returns per-request results and stats."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        small_wait: list[tuple[Req, float]] = []
        large_wait: list[tuple[float, int, Req, float]] = []  # admitted, not started: (cost, order, req, admitted)
        large_run: dict[int, tuple[Req, float, Future]] = {}
        admitted_count = 0
        batch_fut: Optional[Future] = None
        batch_reqs: list[tuple[Req, float]] = []
        used = 0
        results: list[Result] = []
        t0 = self.clock()
        batch_exec = ThreadPoolExecutor(max_workers=1)
        launches = 0

        def now():
            return self.clock() - t0

        while pending or small_wait or large_wait or large_run or batch_fut is not None:
            t = now() if realtime else float("inf")
            progressed = False
            # admission: first come first served while the footprint fits
            while pending and pending[0].arrival <= t:
                r = pending[0]
                need = footprint_bytes(r.n, self.dtype, self.batch_max_n)
                if need > self.budget:
                    raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
                if used + need > self.budget:
                    break
                pending.popleft()
                used += need
                ta = now() if realtime else r.arrival
                if r.n <= self.batch_max_n:
                    small_wait.append((r, ta))
                else:
                    cost = work_estimate(r) if self.large_order == "shortest" else 0.0
                    large_wait.append((cost, admitted_count, r, ta))
                admitted_count += 1
                progressed = True
            # start admitted large requests, shortest estimated work first (or in arrival order)
            while large_wait and len(large_run) < self.large_workers:
                k = min(range(len(large_wait)), key=lambda j: (large_wait[j][0], large_wait[j][1]))
                _, _, r, ta = large_wait.pop(k)
                large_run[r.rid] = (r, ta, self.pool.submit(self.backend.run_large, r))
                progressed = True
            # continuous batching: waiting small requests join the next launch, in
            # arrival order, up to max_launch_shots shots (at least one request)
            if batch_fut is None and small_wait:
                take, shots = 0, 0
                while take < len(small_wait) and (take == 0 or shots + small_wait[take][0].shots <= self.max_launch_shots):
                    shots += small_wait[take][0].shots
                    take += 1
                batch_reqs, small_wait = small_wait[:take], small_wait[take:]
                batch_fut = batch_exec.submit(self.backend.run_batch, [r for r, _ in batch_reqs])
                launches += 1
                progressed = True
            if batch_fut is not None and batch_fut.done():
                out = batch_fut.result()
                tf = now()
                for r, ta in batch_reqs:
                    results.append(Result(r.rid, out[r.rid], r.arrival, ta, tf if realtime else ta, "batch"))
                batch_fut, batch_reqs = None, []
                progressed = True
            for rid in [k for k, (_, _, f) in large_run.items() if f.done()]:
                r, ta, f = large_run.pop(rid)
                cregs = f.result()
                used -= footprint_bytes(r.n, self.dtype, self.batch_max_n)
                tf = now()
                results.append(Result(r.rid, cregs, r.arrival, ta, tf if realtime else ta, "large"))
                progressed = True
            if not realtime and not progressed and pending and not large_run and not large_wait and batch_fut is None:
                raise RuntimeError("admission stalled")
            if not progressed:
                time.sleep(idle_sleep)
        batch_exec.shutdown()
        wall = now()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        shots = int(sum(len(r.cregs) for r in results))
        stats = {
            "requests": len(results), "shots": shots, "wall_s": wall,
            "shots_per_s": shots / wall if wall > 0 else 0.0,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "batched_launches": launches,
            "offered_span_s": max((r.arrival for r in requests), default=0.0),
        }
        return sorted(results, key=lambda r: r.rid), stats

    def close(self):
        self.pool.shutdown()


def serve_sequential(backend, requests: list[Req], clock: Callable[[], float] = time.perf_counter):
    """Baseline: one request at a time in arrival order, all on the plain path
    (one trajectory per shot)."""
    run = getattr(backend, "run_plain", backend.run_large)
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = clock()
    results = []
    for r in reqs:
        while clock() - t0 < r.arrival:
            time.sleep(1e-4)
        ta = clock() - t0
        cregs = run(r)
        results.append(Result(r.rid, cregs, r.arrival, ta, clock() - t0, "plain"))
    wall = clock() - t0
    lat = np.array([r.latency for r in results])
    shots = int(sum(len(r.cregs) for r in results))
    return sorted(results, key=lambda r: r.rid), {
        "requests": len(results), "shots": shots, "wall_s": wall, "shots_per_s": shots / wall,
        "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
    }


def requests_from_stream(stream) -> list[Req]:
    """Converts workloads.serving_stream() output to server requests."""
    return [Req(q.rid, q.arrival, q.n, q.circuit.ops, q.shots) for q in stream]
