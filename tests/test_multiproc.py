"""World-size-2 gloo run of the replica host logic used by bench.py under
torchrun (no GPU): sharding is disjoint and complete, the timing reduction
takes the slowest rank, and the job rate counts every rank's work."""
import os
import socket

import pytest

from paper_2301_06763_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = list(range(13))
        mine = replicas.shard(items, rank, world)
        dist.barrier()
        elapsed = 1.0 + rank            # the slower rank decides
        tmax = replicas.max_over_ranks(elapsed, dist)
        units = replicas.sum_over_ranks(len(mine), dist)
        out.put((rank, mine, tmax, units, replicas.job_rate(units, tmax)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [r[1] for r in res]
    assert sorted(shares[0] + shares[1]) == list(range(13))
    assert not set(shares[0]) & set(shares[1])
    for (_, _, tmax, units, rate) in res:
        assert tmax == 2.0 and units == 13 and rate == 6.5


def test_single_process_helpers():
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        replicas.shard([1], 2, 2)
    with pytest.raises(ValueError):
        replicas.job_rate(1, 0)
