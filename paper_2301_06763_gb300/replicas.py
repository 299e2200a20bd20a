"""Host logic of multi-GPU runs: replicas, no data-path collective.

Meshes (and the levels inside one) are independent sub-problems (Sect. 4 of
the paper), so N GPUs each solve their own share: a batch is sharded
round-robin, a single-mesh benchmark runs one replica per rank (weak scaling).
The only communication is timing: a barrier before and after the timed region
and the maximum elapsed time over ranks.
"""


def shard(items, rank, world):
    """Round-robin share of ``items`` for ``rank`` of ``world`` (disjoint, complete)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world %r/%r" % (rank, world))
    return list(items)[rank::world]


def max_over_ranks(value, dist=None, device=None):
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device=None):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(total_units, max_elapsed_s):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    if max_elapsed_s <= 0:
        raise ValueError("elapsed time must be positive")
    return total_units / max_elapsed_s
