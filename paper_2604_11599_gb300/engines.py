"""One entry point for shots of a program, choosing the engine.

* ``clifford`` -- stabilizer tableaux (``sv.Clifford``), for programs whose
  gates are all Clifford on at most 64 qubits;
* ``batched``  -- the persistent batched launch with shot branching
  (``sv.Batch.sample_branched``), for programs of at most ``batch_max_n``
  qubits (each trajectory runs inside one CTA);
* ``plain``    -- the resident-state path with shot branching
  (``sv.State.sample_branched``), for everything else.

The state-vector engines give every shot the record its own trajectory gives;
the tableaux give the same records except where a state vector's rounded
p0/(p0+p1) and 1/2 straddle the shot's Philox number.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from .ir import Gate, Kind

CLIFFORD_GATES = frozenset({Gate.I, Gate.H, Gate.X, Gate.Y, Gate.Z, Gate.S, Gate.SDG, Gate.SX, Gate.CX, Gate.CY,
                            Gate.CZ, Gate.SWAP})


def is_clifford(ops: np.ndarray) -> bool:
    """Every gate record is in the tableau engine's gate set and no record is dense."""
    kinds = ops["kind"]
    if (kinds == int(Kind.DENSE)).any():
        return False
    gates = ops["gate"][kinds == int(Kind.GATE)]
    return all(int(g) in CLIFFORD_GATES for g in np.unique(gates))


def choose(ops: np.ndarray, n: int, params=None, pool=None, batch_max_n: int = 20) -> str:
    """The engine ``sample`` uses for this program."""
    has_params = params is not None and len(params) and (ops["pidx"] >= 0).any()
    if n <= 64 and is_clifford(ops) and not has_params and (pool is None or not len(pool)):
        return "clifford"
    if n > 34:
        raise ValueError(f"{n} qubits: only Clifford programs run beyond 34 qubits")
    return "batched" if n <= batch_max_n else "plain"


def sample(ops: np.ndarray, n: int, shots: int, dtype: str = "c64", params=None, pool=None, seed: int = 0,
           stream_id: int = 0, engine: str = "auto", batch_max_n: int = 20) -> tuple[np.ndarray, dict]:
    """Registers of shots 0..shots-1 and a dict naming the engine (plus the
    branching statistics of the state-vector engines)."""
    from . import sv

    ops = np.ascontiguousarray(ops)
    eng = choose(ops, n, params, pool, batch_max_n) if engine == "auto" else engine
    if eng == "clifford":
        with sv.Clifford(n, ops) as h:
            return h.sample(shots, seed=seed, stream_id=stream_id), {"engine": "clifford"}
    if eng == "batched":
        with sv.Batch(dtype) as b:
            p = b.add_program(ops, n, params=params, pool=pool)
            regs, st = b.sample_branched([p], [stream_id], [shots], seed=seed)
        return regs, {"engine": "batched", **st}
    if eng == "plain":
        with sv.State(n, dtype) as s:
            if pool is not None and len(pool):
                s.set_dense_pool(pool)
            regs, st = s.sample_branched(ops, shots, params=params, seed=seed, stream_id=stream_id)
        return regs, {"engine": "plain", **st}
    raise ValueError(f"unknown engine {engine!r}")


__all__ = ["CLIFFORD_GATES", "is_clifford", "choose", "sample"]
