"""Work division across processes (one process per GPU).

A single solve does not shard: every smoothing colour on every level would
need a halo exchange.  Independent grids (a batch) and independent requests
do: each rank takes a share of the grids, chosen by longest-processing-time
first on the cell count, and no data moves between ranks; only the timing
(slowest rank) and the per-grid statuses are gathered on the host side.
"""
from __future__ import annotations

import heapq


def partition_lpt(costs, world: int):
    """Indices of ``costs`` for each of ``world`` ranks, by longest
    processing time first: the largest remaining item goes to the least
    loaded rank (ties to the lower rank).  Deterministic, so every rank
    computes the same division without communicating.  The heaviest share
    is at most 4/3 of the best possible."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def max_over_ranks(value: float, device=None) -> float:
    """The largest ``value`` over all ranks (the job's time is its slowest
    rank's); the value itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_statuses(share, statuses, world: int):
    """Every rank's (grid index, status) pairs merged into one list in grid
    order (host objects only)."""
    import torch.distributed as dist
    mine = list(zip(share, [int(s) for s in statuses]))
    if world == 1 or not dist.is_initialized():
        return [s for _, s in sorted(mine)]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    merged = sorted(p for part in parts for p in part)
    return [s for _, s in merged]
