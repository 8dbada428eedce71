"""Multi-GPU host logic on CPU: world-size-2 gloo ranks (no GPU)."""
import os
import socket

import pytest

from paper_2207_12244_gb300 import replicas


def test_shard_covers_every_item_once():
    for n in (0, 1, 5, 64, 101):
        for world in (1, 2, 3, 8):
            owned = [replicas.shard(n, r, world) for r in range(world)]
            flat = sorted(i for o in owned for i in o)
            assert flat == list(range(n))
            sizes = [len(o) for o in owned]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(10, rank, world)
        # per-rank "time" and "units": the job's time is the slowest rank's,
        # the job's units are everybody's
        t = replicas.max_over_ranks(1.5 + rank)
        u = replicas.sum_over_ranks(len(mine))
        q.put((rank, mine, t, u, replicas.rank_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_reduce():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, u0, s0), (r1, m1, t1, u1, s1) = res
    assert m0 == [0, 1, 2, 3, 4] and m1 == [5, 6, 7, 8, 9]
    assert t0 == t1 == 2.5
    assert u0 == u1 == 10
    assert s0 != s1
