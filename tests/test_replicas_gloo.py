"""The multi-GPU path is replicas: ranks shard independent units and combine
only their timing.  Two gloo ranks on CPU check the host logic that bench.py
uses for N > 1 (sharding, independent draw streams, max over ranks, whole-job
rate)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_11599_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = list(replicas.shard(10, rank, world))
        local_seconds = 1.0 + rank  # rank 1 is the slow one
        slowest = replicas.max_over_ranks(local_seconds, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, units)
        rate = replicas.whole_job_rate(float(len(units)), slowest, world)
        out[rank] = (units, replicas.stream_of(rank), slowest, gathered, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    u0, s0, m0, g0, r0 = out[0]
    u1, s1, m1, g1, r1 = out[1]
    assert sorted(u0 + u1) == list(range(10)) and not set(u0) & set(u1)
    assert s0 != s1
    assert m0 == m1 == 2.0
    assert g0 == g1 == [u0, u1]
    assert r0 == pytest.approx(5 * 2 / 2.0)


def test_single_process_fallbacks():
    assert list(replicas.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate([3.0, 5.0], 2.0) == 4.0
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
