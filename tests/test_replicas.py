"""Host logic of the multi-GPU mode (independent replicas), with two gloo ranks on
the CPU: sharding of independent solves and the job-level throughput."""
import os
import socket

import pytest

from paper_1701_07559_gb300 import replicas


def test_shard_covers_every_item_once():
    for n in (0, 1, 5, 12, 300):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in replicas.shard(n, r, world))
            assert got == list(range(n))
            sizes = [len(replicas.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_reductions():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.job_throughput(12, 2.0) == 6.0


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        mine = replicas.shard(12, rank, world)
        # rank r pretends to have solved its share in (r + 1) seconds
        thr = replicas.job_throughput(len(mine), float(rank + 1), dist)
        q.put((rank, mine, thr, replicas.max_over_ranks(rank + 1, dist), replicas.sum_over_ranks(len(mine), dist)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, mx0, s0), (r1, m1, t1, mx1, s1) = out
    assert sorted(m0 + m1) == list(range(12))
    assert mx0 == mx1 == 2.0 and s0 == s1 == 12.0
    assert t0 == t1 == pytest.approx(12 / 2.0)
