"""Work split over GPUs.

Independent removals (images, requests) shard with no collective on the data
path: every rank computes the same deterministic assignment from the same
work estimates and takes its own share; the only cross-rank operation is the
max of the timed region that a benchmark reports.

One removal can also be split over ranks by candidate rows (run_row_sharded):
each rank holds a full replica of the removal state, searches its slab of
candidate rows (findBestPatch, Sec. 3, Eq. 3-4, is a minimum over candidate
centres), one all-reduce-min of the 8-byte packed key per iteration picks the
global source patch, and every replica applies it, so the replicas stay
identical with no other exchange.
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


# -- one removal split over ranks by candidate rows ---------------------

KEY_NONE = (1 << 64) - 1   # no candidate in the searched rows
_I64_MAX = (1 << 63) - 1


def row_slabs(y0: int, y1: int, world: int):
    """Contiguous half-open row ranges, one per rank, covering the candidate
    rows [y0, y1] (inclusive) with sizes that differ by at most one (empty
    ranges when there are fewer rows than ranks)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = max(0, y1 - y0 + 1)
    return [(y0 + k * n // world, y0 + (k + 1) * n // world) for k in range(world)]


def min_key_over_ranks(key: int) -> int:
    """Minimum of a packed key (SSD << 32 | index) over the ranks of the
    default process group.  Real keys are below 2^63 (an SSD of at most
    65 * 65 * 3 * 255^2 < 2^31), so they reduce as int64, KEY_NONE standing
    in as the int64 maximum."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(key)
    v = _I64_MAX if key == KEY_NONE else int(key)
    if not 0 <= v <= _I64_MAX:
        raise ValueError(f"key {key:#x} out of range")
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    v = int(t.item())
    return KEY_NONE if v == _I64_MAX else v


def run_row_sharded(replica, rank: int | None = None, world: int | None = None,
                    reduce=min_key_over_ranks, max_iters: int = 0):
    """Runs one removal with the search split over ranks by candidate rows.

    `replica` is this rank's copy of the removal (every rank starts from the
    same inputs) with search_rect() -> (x0, x1, y0, y1), search_rows(y0, y1)
    -> smallest key of those rows (KEY_NONE if none; None once the removal
    is done) and apply_key(key) -> the iteration's record.  Each iteration
    searches this rank's slab, reduces the key over the ranks and applies
    the result.  Returns this rank's records (identical on every rank)."""
    if rank is None or world is None:
        import torch.distributed as dist

        on = dist.is_available() and dist.is_initialized()
        rank = dist.get_rank() if on else 0
        world = dist.get_world_size() if on else 1
    _, _, y0, y1 = replica.search_rect()
    lo, hi = row_slabs(y0, y1, world)[rank]
    recs = []
    while max_iters <= 0 or len(recs) < max_iters:
        key = replica.search_rows(lo, hi)
        if key is None:
            break  # every replica is in the same state: all ranks stop together
        recs.append(replica.apply_key(reduce(key)))
    return recs
