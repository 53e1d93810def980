"""Sharding of independent GBP problems across ranks (one GPU per rank).

Independent problems share no variable, so a batch shards with no exchange
on the data path: each rank solves its own subset in one graph, and the
ranks meet only to agree on timing.  The subsets are balanced by size with
the longest-processing-time rule (largest problem first, each to the rank
with the least work so far; ties to the lowest rank), which bounds the
busiest rank at 4/3 of the optimum.
"""
from __future__ import annotations

import heapq


def partition(sizes, n_ranks: int):
    """Split problem indices 0..len(sizes)-1 over n_ranks by size.

    Returns a list of n_ranks ascending index lists; deterministic for given
    sizes (ties in size keep index order)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(n_ranks)]
    out = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(x) for x in out]


def loads(sizes, parts):
    return [sum(int(sizes[i]) for i in p) for p in parts]


def reduce_timing(ms: float, units: float, device=None):
    """Whole-job figures over the ranks of the default process group: the
    slowest rank's time (max) and the units of work of all ranks (sum).
    Without an initialised process group, returns the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
