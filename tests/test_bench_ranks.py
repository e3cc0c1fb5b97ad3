"""The replica path of bench.py with N > 1 ranks (one process per GPU there):
the whole-job time is the slowest rank's and the node updates add up.  Run
here as two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t, u = bench.job_totals(torch, 10.0 + 5.0 * rank, 1000 * (rank + 1), world, torch.device("cpu"))
        q.put((rank, t, u))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_sum_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1:] for r in res] == [(15.0, 3000.0), (15.0, 3000.0)]


def test_one_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(torch, 7.5, 42, 1, None) == (7.5, 42.0)
