"""The multi-GPU replica path's host logic on CPU: two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2212_14153_gb300 import replicas


def test_shard_covers_every_item_once():
    items = list(range(17))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        replicas.shard(items, 3, 3)


def test_single_process_reductions_are_identity():
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.job_rate(100.0, 4.0) == 25.0


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = replicas.shard(list(range(10)), rank, world)
        units = float(sum(work))            # rank 0: 0+2+..+8 = 20, rank 1: 25
        secs = 1.0 + rank                   # rank 1 is the slowest
        out[rank] = (replicas.max_over_ranks(secs), replicas.sum_over_ranks(units),
                     replicas.job_rate(units, secs))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_combine_time_and_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        mx, tot, rate = out[r]
        assert mx == 2.0 and tot == 45.0 and rate == 22.5
