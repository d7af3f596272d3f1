"""Host-side logic of the multi-GPU path: independent runs, no data-path collective.

The method's parallelism is independent deposition runs (the paper's dataset is a
sweep of runs, "Dataset"), so N GPUs either run N replicas of a workload or
split an ensemble's run list.  The only collectives are on timings and counts.
"""
from __future__ import annotations


def shard_runs(costs, world_size: int, rank: int) -> list[int]:
    """Indices of the runs rank `rank` takes: greedy longest-processing-time split by
    cost (cells x steps), deterministic on every rank, every run on exactly one rank."""
    if world_size < 1 or not (0 <= rank < world_size):
        raise ValueError("bad world size or rank")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world_size
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def aggregate(seconds: float, units: float, group=None, device=None) -> tuple[float, float]:
    """(max seconds over ranks, total units over ranks); the whole-job throughput is
    total / max.  Without an initialised process group this is the identity."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds), float(units)
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
