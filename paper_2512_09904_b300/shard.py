"""Whole-case sharding of a sweep over the ranks of one node.

Cases are independent problems: each rank runs its own share in its own
batch on its own GPU, and only the per-case results travel, on the host, to
rank 0.  There is no data-path collective.

    assign_cases(sizes, world)   -> rank of every case (largest first, to the
                                    rank with the fewest particles so far)
    gather_results(local, ...)   -> rank 0: every rank's {case index: result}
    reduce_timing(ms, units)     -> (max ms over ranks, sum of units): the
                                    whole-job throughput of a timed region
"""
from __future__ import annotations

import heapq


def assign_cases(sizes, world):
    """Greedy longest-first assignment of case sizes (particle counts) to
    `world` ranks: deterministic (ties broken by case index, then rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    rank_of = [0] * len(sizes)
    for i in order:
        load, r = heapq.heappop(heap)
        rank_of[i] = r
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return rank_of


def gather_results(local, rank, world, group=None):
    """Merge per-rank dicts {case index: result} on rank 0 (host objects over
    the process group); other ranks get None."""
    import torch.distributed as dist
    if world == 1:
        return dict(local)
    parts = [None] * world if rank == 0 else None
    dist.gather_object(local, parts, dst=0, group=group)
    if rank != 0:
        return None
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"case {k} reported by two ranks")
            merged[k] = v
    return merged


def reduce_timing(ms, units, world, device=None):
    """Whole-job timing of one timed region: the slowest rank's time and the
    units every rank processed.  Returns (ms_max, units_sum)."""
    if world == 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms), float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])
