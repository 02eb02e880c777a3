"""Host-side logic of the multi-GPU runs: one process per GPU, independent problems per rank.

The sweep shards by independent problems: every group (and every whole instance) is swept without data from
any other, so ranks never exchange data on the path.  The only collectives are the timing ones: a barrier
around the timed region and the maximum of the per-rank times.  Works with any torch.distributed backend
(NCCL on GPUs, gloo on CPU for the tests).
"""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_seed(base: int, rank: int) -> int:
    """Seed of the instance a rank sweeps in a weak-scaling run (each rank its own seeded instance)."""
    return base + rank


def shard_groups(G: int, world: int, rank: int) -> range:
    """Contiguous group range of a rank when one instance is split by groups: sizes differ by at most one
    (every group costs the same number of updates), lower ranks take the extra groups."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(G, world)
    g0 = rank * q + min(rank, r)
    return range(g0, g0 + q + (1 if rank < r else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (the timed region's duration) over all ranks; the value itself when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max
