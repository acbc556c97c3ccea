"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the batch
instances are dealt to the ranks with every instance on exactly one rank, and
the job time is the slowest rank's."""
import os
import socket

import pytest

import pf_inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plist = I.batch_manifest(count=13)
    mine = bench.deal(plist, rank, world)
    # a rank-dependent "time": the job time must be the largest
    t = bench.job_time(1.0 + rank * 0.5, dist, "cpu")
    out.put((rank, [plist.index(p) for p in mine], t))
    dist.destroy_process_group()


def test_deal_and_max_time_two_ranks():
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
    res.sort()
    got = sorted(i for _, idx, _ in res for i in idx)
    assert got == list(range(13))                      # every instance once
    assert set(res[0][1]).isdisjoint(res[1][1])
    assert [len(r[1]) for r in res] == [7, 6]          # dealt i mod 2
    assert all(abs(t - 1.5) < 1e-12 for _, _, t in res)   # max over ranks


def test_deal_single_rank_is_identity():
    import bench

    items = list(range(5))
    assert bench.deal(items, 0, 1) == items
    assert bench.job_time(2.5) == 2.5
