"""Host logic of multi-GPU runs: independent replicas and instance sharding.

One process per GPU.  A single transport problem is never split across GPUs (one
iteration at 256 x 256 costs less than an inter-GPU halo exchange); independent
problems are.  Nothing here touches the solver's data path: the only collectives
are the scalar reductions of a benchmark's timing and the optional gather of
per-instance results.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world size, local rank) from the torchrun environment (0, 1, 0 without it)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_instances(weights, world: int):
    """Split instances over `world` ranks by estimated cost (longest first, each to the
    least-loaded rank; ties to the lowest rank).  Returns one sorted index list per rank;
    every index appears exactly once.  Deterministic, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda q: (-float(weights[q]), q))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for q in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(q)
        load[r] += float(weights[q])
    return [sorted(p) for p in parts]


def instance_weight(n: int, k: int, l: int, iters: int = 1):
    """Estimated cost of one instance: algorithmic bytes 4(7k + 2l) per point and iteration."""
    return 4.0 * (7 * k + 2 * l) * n * n * iters


def aggregate_throughput(local_ms: float, local_units: float, dist=None, device=None):
    """Whole-job time and work: the slowest rank's time and the sum of all ranks' units
    (weak scaling: every rank runs its own replica).  `dist` is torch.distributed when a
    process group is up, else None (one process)."""
    if dist is None:
        return float(local_ms), float(local_units)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
