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
