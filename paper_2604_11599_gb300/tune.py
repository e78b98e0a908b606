"""Autotuner: the planner's tuning and the kernel variant, chosen by timing.

For a program class on this GPU -- qubit count, dtype and the program's
structure (record kinds, gates, qubits, control flow and parameter slots, not
its literal angles) -- the tuner times candidate settings on the real kernels
and keeps the fastest in a JSON cache keyed by (device name, SM count, n,
dtype, structure), so later runs of the same class pay nothing.

* Plain path (``sv_set_tuning``, ``sv_set_jit``): tile bits (tiles of 2^10 to
  2^14 amplitudes), contiguous low qubits of a tile, gates fused into one pass
  (0: as many as the planner can), and whether the passes run as kernels
  compiled for the program.
* Batched launch (``sv_batch_set_tuning``): contiguous low qubits and gates
  per pass (the batched kernel fixes the tile at 2^12 amplitudes).

The search itself (``autotune``) takes the timing function as an argument,
so its logic runs without a GPU.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time
from dataclasses import asdict, dataclass
from typing import Callable, Iterable, Optional, Sequence

import numpy as np

from .ir import OP_DTYPE


@dataclass(frozen=True)
class Setting:
    tile_bits: int = 0       # 0: planner default (12)
    low_bits: int = 0        # 0: planner default
    max_pass_gates: int = 0  # 0: planner default (as many as fit)
    jit: bool = False        # passes as kernels compiled for the program

    def label(self) -> str:
        return f"t{self.tile_bits}-l{self.low_bits}-g{self.max_pass_gates}-{'jit' if self.jit else 'gen'}"


def structure_hash(ops: np.ndarray) -> str:
    """Hash of the program without its literal angles: programs that differ only
    in rotation angles or parameter values share a tuning."""
    a = np.ascontiguousarray(ops, dtype=OP_DTYPE).copy()
    if a.size:
        lit = a["pidx"] < 0
        ang = a["angle"]
        ang[lit] = 0.0
        a["angle"] = ang
    return hashlib.sha1(a.tobytes()).hexdigest()[:16]


def plain_candidates(n: int, dtype: str = "c64", ops: Optional[np.ndarray] = None, pool=None,
                     tiles: Sequence[int] = (10, 12, 14), lows: Sequence[int] = (3, 4, 6),
                     gates: Sequence[int] = (0,), jit: Sequence[bool] = (False, True)) -> list[Setting]:
    """Settings the planner accepts for n qubits (tiles no larger than the state
    nor than shared memory allows for the dtype: 2^13 complex128 amplitudes;
    tile_bits - low_bits <= 9); with `ops`, each is planned on the host
    (sv_plan_info) and kept as the tile and low bits the planner actually used,
    duplicates dropped."""
    n_int = max(n, 10)
    t_max = 14 if dtype == "c64" else 13
    out = []
    for t in tiles:
        if t > n_int or t > t_max:
            continue
        for lo in lows:
            if not (2 <= lo <= t and t - lo <= 9):
                continue
            for g in gates:
                for j in jit:
                    out.append(Setting(t, lo, g, bool(j)))
    if ops is not None:
        from . import sv

        ok, seen = [], set()
        for s in out:
            try:
                st = sv.plan_info(ops, n, dtype, pool, s.tile_bits, s.low_bits, s.max_pass_gates)
            except sv.SVError:
                continue
            e = Setting(int(st["tile_bits"]), int(st["low_bits"]), s.max_pass_gates, s.jit)
            if e not in seen:
                seen.add(e)
                ok.append(e)
        out = ok
    return out


def batch_candidates(lows: Sequence[int] = (0,), gates: Sequence[int] = (0, 8, 16, 32)) -> list[Setting]:
    """Batched-launch settings (tile fixed at 12 bits; low bits 3..12 or 0 for the
    default).  By default only the fusion width varies: it changes the plan the
    kernel runs, not the kernel's tile geometry."""
    return [Setting(12, lo, g, False) for lo in lows if lo == 0 or 3 <= lo <= 12 for g in gates]


def autotune(measure: Callable[[Setting], float], candidates: Iterable[Setting], reps: int = 3,
             errors: tuple = ()) -> tuple[Setting, dict]:
    """Times every candidate `reps` times (median) and returns the fastest with
    the table of medians.  Candidates whose measurement raises one of `errors`
    are left out; if none is left, RuntimeError."""
    table: dict[Setting, float] = {}
    for s in candidates:
        try:
            ts = [float(measure(s)) for _ in range(max(1, reps))]
        except errors:
            continue
        table[s] = statistics.median(ts)
    if not table:
        raise RuntimeError("no candidate setting could be measured")
    best = min(table, key=lambda s: (table[s], s.label()))
    return best, table


class Cache:
    """JSON file of tuned settings: {key: {"setting": {...}, "ms": {label: ms}}}."""

    def __init__(self, path: Optional[str] = None):
        self.path = path or os.environ.get("SV_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "paper_2604_11599_gb300", "tune.json")
        self.data: dict = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str) -> Optional[Setting]:
        e = self.data.get(key)
        return Setting(**e["setting"]) if e else None

    def put(self, key: str, setting: Setting, table: Optional[dict] = None) -> None:
        self.data[key] = {"setting": asdict(setting),
                          "ms": {s.label(): v for s, v in (table or {}).items()}}

    def save(self) -> None:
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def device_tag() -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}sm"


def apply(state, s: Setting) -> None:
    """Puts a plain-path setting on a sv.State."""
    state.set_tuning(s.tile_bits, s.low_bits, s.max_pass_gates)
    state.set_jit(s.jit)


def time_plain(ops: np.ndarray, n: int, dtype: str, s: Setting, params=None, pool=None, seed: int = 0) -> float:
    """Milliseconds of one run of the prepared program with setting s (CUDA
    events on the state's stream, after one warm-up run)."""
    import torch

    from . import sv

    with sv.State(n, dtype) as st:
        if pool is not None and len(pool):
            st.set_dense_pool(pool)
        apply(st, s)
        prog = st.prepare(ops)
        dp = None if params is None else torch.as_tensor(np.asarray(params, dtype=np.float64), device="cuda")
        st.launch(prog, dp, seed=seed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.launch(prog, dp, seed=seed)
        e1.record()
        e1.synchronize()
        return float(e0.elapsed_time(e1))


def tune_plain(ops: np.ndarray, n: int, dtype: str = "c64", cache: Optional[Cache] = None,
               candidates: Optional[Sequence[Setting]] = None, reps: int = 3, params=None, pool=None,
               force: bool = False) -> Setting:
    """The cached setting of this program class, or the fastest candidate (timed
    now and cached)."""
    from . import sv

    cache = cache or Cache()
    key = f"plain|{device_tag()}|n{n}|{dtype}|{structure_hash(ops)}"
    if not force:
        hit = cache.get(key)
        if hit is not None:
            return hit
    cands = list(candidates) if candidates is not None else plain_candidates(n, dtype, ops, pool)
    best, table = autotune(lambda s: time_plain(ops, n, dtype, s, params, pool), cands, reps, errors=(sv.SVError,))
    cache.put(key, best, table)
    cache.save()
    return best


def time_batch(programs: Sequence[tuple], dtype: str, s: Setting, n_items: int = 2048, seed: int = 0) -> float:
    """Milliseconds of one batched launch of n_items trajectories spread over
    `programs` ((ops, n) pairs) with setting s, after one warm-up launch."""
    from . import sv

    with sv.Batch(dtype) as b:
        b.set_tuning(s.low_bits, s.max_pass_gates)
        ids = [b.add_program(ops, n) for ops, n in programs]
        prog = np.array([ids[i % len(ids)] for i in range(n_items)], dtype=np.uint32)
        b.set_items(prog, np.arange(n_items), np.zeros(n_items))
        b.launch(seed)
        b.results()
        t0 = time.perf_counter()
        b.launch(seed)
        b.results()
        return 1000.0 * (time.perf_counter() - t0)


def tune_batch(programs: Sequence[tuple], dtype: str = "c64", cache: Optional[Cache] = None,
               candidates: Optional[Sequence[Setting]] = None, reps: int = 3, n_items: int = 2048,
               force: bool = False) -> Setting:
    """The cached or freshly timed batched-launch setting for this mix of
    (ops, n) programs; apply it with Batch.set_tuning(s.low_bits, s.max_pass_gates)
    before adding the programs."""
    from . import sv

    cache = cache or Cache()
    sig = hashlib.sha1("|".join(f"{n}:{structure_hash(ops)}" for ops, n in programs).encode()).hexdigest()[:16]
    key = f"batch|{device_tag()}|{dtype}|{sig}"
    if not force:
        hit = cache.get(key)
        if hit is not None:
            return hit
    cands = list(candidates) if candidates is not None else batch_candidates()
    best, table = autotune(lambda s: time_batch(programs, dtype, s, n_items), cands, reps, errors=(sv.SVError,))
    cache.put(key, best, table)
    cache.save()
    return best


__all__ = ["Setting", "structure_hash", "plain_candidates", "batch_candidates", "autotune", "Cache", "device_tag",
           "apply", "time_plain", "tune_plain", "time_batch", "tune_batch"]
