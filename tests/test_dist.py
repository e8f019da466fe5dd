"""Rank sharding of independent removals and the max-over-ranks timing, with
two gloo ranks on the CPU (the multi-GPU path has no data-path collective)."""
import os
import socket

import pytest

from paper_1403_4238_gb300 import dist as pdist


def test_shard_by_work_covers_every_item_once_and_balances():
    works = [float((i * 37) % 11 + 1) for i in range(64)]
    for world in (1, 2, 3, 8):
        parts = pdist.shard_by_work(works, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(works[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(works)  # LPT bound
    assert pdist.shard_by_work([], 2) == [[], []]
    with pytest.raises(ValueError):
        pdist.shard_by_work([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        works = [float(w) for w in range(1, 41)]
        mine = pdist.my_share(works, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = pdist.max_over_ranks(10.0 + rank)
        q.put((rank, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_split_and_max():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, t in res:
        assert t == 11.0
        assert sorted(i for part in got for i in part) == list(range(40))
        assert not set(got[0]) & set(got[1])
    assert res[0][1] == res[1][1]


# -- one removal split over ranks by candidate rows ----------------------

STEP_FIELDS = ("px", "py", "qx", "qy", "ssd", "filled", "remaining")


def test_row_slabs_partition_the_rows():
    for y0, y1 in ((4, 91), (4, 4), (10, 9)):
        for world in (1, 2, 3, 5, 200):
            slabs = pdist.row_slabs(y0, y1, world)
            assert len(slabs) == world
            rows = [y for lo, hi in slabs for y in range(lo, hi)]
            assert rows == list(range(y0, y1 + 1))
            sizes = [hi - lo for lo, hi in slabs]
            assert max(sizes) - min(sizes) <= 1


def test_min_over_row_slabs_is_the_full_search():
    """Replicas that search disjoint slabs and apply the minimum key follow
    the oracle's own run, iteration by iteration (3 emulated ranks, one of
    them with a slab that starts above the search rectangle)."""
    import numpy as np

    import oracle
    from oracle_replica import OracleReplica
    from paper_1403_4238_gb300 import synth

    case = synth.small_rect(seed=71)
    full = oracle.run(case.rgb, case.mask, case.r)
    reps = [OracleReplica(case.rgb, case.mask, case.r) for _ in range(3)]
    _, _, y0, y1 = reps[0].search_rect()
    slabs = pdist.row_slabs(y0, y1, 3)
    slabs[0] = (0, slabs[0][1])
    recs = []
    while True:
        keys = [rep.search_rows(lo, hi) for rep, (lo, hi) in zip(reps, slabs)]
        if keys[0] is None:
            assert all(k is None for k in keys)
            break
        g = min(keys)
        out = [rep.apply_key(g) for rep in reps]
        assert all(o[f] == out[0][f] for o in out for f in STEP_FIELDS)
        recs.append(out[0])
    assert len(recs) == full.iters
    for a, b in zip(recs, full.trace):
        assert all(a[f] == b[f] for f in STEP_FIELDS)
    for rep in reps:
        assert np.array_equal(rep.rgb, full.rgb)


def _sharded_worker(rank, world, port, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(__file__))
    from oracle_replica import OracleReplica
    from paper_1403_4238_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = synth.small_rect(seed=72)
        rep = OracleReplica(case.rgb, case.mask, case.r)
        recs = pdist.run_row_sharded(rep)
        q.put((rank, [tuple(int(t[f]) for f in STEP_FIELDS) for t in recs], rep.rgb.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_one_removal_row_sharded():
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    from paper_1403_4238_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = synth.small_rect(seed=72)
    full = oracle.run(case.rgb, case.mask, case.r)
    want = [tuple(int(t[f]) for f in STEP_FIELDS) for t in full.trace]
    for rank, recs, rgb in res:
        assert recs == want
        assert np.frombuffer(rgb, np.uint8).reshape(full.rgb.shape).tolist() == full.rgb.tolist()


def _minkey_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        k = (32967075 << 32) | 5 if rank == 0 else (7 << 32) | 123456
        got = [
            pdist.min_key_over_ranks(k),                                      # both real
            pdist.min_key_over_ranks(pdist.KEY_NONE if rank else (9 << 32)),  # one side has none
            pdist.min_key_over_ranks(pdist.KEY_NONE),                         # nobody has one
            pdist.min_key_over_ranks((3 << 32) | (10 + rank)),                # SSD tie: lower index
        ]
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_min_key_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_minkey_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got in res:
        assert got == [(7 << 32) | 123456, 9 << 32, pdist.KEY_NONE, (3 << 32) | 10]
