"""Multi-GPU by replicas: the simulated work shards into independent units
(trajectories, shots, parameter sets, requests) with no exchange between
them, so N processes, one per GPU, each run their own share and only the
timing is combined.  No collective touches the data path.

These helpers are the host-side logic of that scheme (they run with any
``torch.distributed`` backend, gloo included):

* ``shard``        -- the units of one rank (round-robin, every unit exactly once);
* ``stream_of``    -- the Philox stream id of a rank's trajectories, so that
                      ranks draw independent outcomes;
* ``max_over_ranks`` -- the slowest rank's time, which a whole-job rate divides by.
"""
from __future__ import annotations

from typing import Optional, Sequence


def shard(n_units: int, rank: int, world: int) -> range:
    """Unit indices of ``rank`` out of ``world``: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return range(rank, n_units, world)


def stream_of(rank: int, base: int = 0) -> int:
    """Philox stream id of a rank's trajectories (key = (seed, stream))."""
    return base + rank


def max_over_ranks(value: float, dist=None, device: Optional[str] = None) -> float:
    """The largest ``value`` over the ranks of the default process group
    (``value`` itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: Sequence[float] | float, seconds_max: float, world: int = 1) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    total = sum(units_per_rank) if isinstance(units_per_rank, Sequence) else float(units_per_rank) * world
    return total / seconds_max
