"""Work split over GPUs for independent removals (replicas, no collective on
the data path).

A removal is a strict sequence of iterations on one image, so GPUs share
work only at the granularity of whole images or requests.  Every rank
computes the same deterministic assignment from the same work estimates and
takes its own share; the only cross-rank operation is the max of the timed
region that a benchmark reports.
"""
from __future__ import annotations

import heapq


def shard_by_work(works, world: int):
    """Longest-processing-time-first assignment of items (estimated work
    each) to `world` ranks; returns one sorted index list per rank.  Ties go
    to the lower rank, so every rank derives the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(works[i]), r))
    return [sorted(x) for x in out]


def my_share(works, rank: int, world: int):
    return shard_by_work(works, world)[rank]


def max_over_ranks(value: float) -> float:
    """Max of a float over the ranks of the default process group (the value
    itself when no group is initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
