"""The multi-rank bookkeeping of bench.py (paper_2309_08235_gb300.replicas)
on CPU with world size 2 over gloo: disjoint shares that cover a problem set,
the barrier, and the whole-job rate = summed units / slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2309_08235_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = R.env()
        items = list(R.shard(256, r, w))
        R.barrier(dist)
        # rank r "processed" its items at 10 units each in (1 + r) seconds
        rate, tmax, total = R.job_rate(10.0 * len(items), 1.0 + r, dist)
        out.put((r, items, rate, tmax, total))
    finally:
        dist.destroy_process_group()


def test_shard_covers_once():
    for n in (0, 1, 7, 256, 1001):
        for w in (1, 2, 3, 8):
            got = [i for r in range(w) for i in R.shard(n, r, w)]
            assert got == list(range(n))
            sizes = [len(R.shard(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.shard(10, 2, 2)


def test_single_process_rate():
    assert R.job_rate(100.0, 2.0) == (50.0, 2.0, 100.0)


def test_two_ranks_over_gloo():
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
    (r0, i0, rate0, t0, u0), (r1, i1, rate1, t1, u1) = res
    assert sorted(i0 + i1) == list(range(256)) and not set(i0) & set(i1)
    # slowest rank: 2 s; all units: 2560 -> 1280 units/s on both ranks
    assert t0 == t1 == 2.0 and u0 == u1 == 2560.0
    assert rate0 == rate1 == 1280.0
