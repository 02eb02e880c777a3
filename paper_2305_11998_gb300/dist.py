"""Host-side logic of the multi-GPU runs: one process per GPU, one instance split by contiguous group ranges.

The sweep shards by groups: every group is swept without data from any other (kappa_g, B_g, its boundary values,
its intensity state and its moments touch no other group), so ranks never exchange data on the path.  A rank
builds a plan over its own group range on the full characteristic grid and sweeps the group slices of the inputs.
The collectives are the timing ones (a barrier around the timed region, the maximum of the per-rank times) and,
for a consumer that needs every group on every GPU (the grey closure), an all-gather of the per-group results.
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU for the tests).
"""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_groups(G: int, world: int, rank: int) -> range:
    """Contiguous group range of a rank when one instance is split by groups: sizes differ by at most one
    (every group costs the same number of updates), lower ranks take the extra groups."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(G, world)
    g0 = rank * q + min(rank, r)
    return range(g0, g0 + q + (1 if rank < r else 0))


def shard_inputs(d: dict, groups: range) -> dict:
    """The group slices of a workload's inputs for one shard: kappa and B rows [g0, g1) of [G][cell], the boundary
    columns [g0, g1) of [4][G] (copied contiguous); c and dt as they are."""
    import numpy as np
    g0, g1 = groups.start, groups.stop
    out = dict(d)
    out["kappa"] = np.ascontiguousarray(d["kappa"][g0:g1])
    out["B"] = np.ascontiguousarray(d["B"][g0:g1])
    out["bnd"] = np.ascontiguousarray(d["bnd"][:, g0:g1])
    return out


def gather_groups(local, G: int, groups: range, world: int, device=None):
    """All-gather of a per-group array [g1 - g0][n] from every rank into the full [G][n] on every rank (ranks hold
    contiguous, ordered group ranges of sizes differing by at most one: each contribution is padded to the largest
    range for the collective)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return local
    n = local.shape[1]
    q, r = divmod(G, world)
    rows = q + (1 if r else 0)
    buf = torch.zeros((rows, n), dtype=local.dtype, device=local.device)
    buf[: local.shape[0]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return torch.cat([parts[k][: len(shard_groups(G, world, k))] for k in range(world)], 0)


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
