"""bench.py's multi-rank bookkeeping on CPU (gloo, world size 2): every rank
ends with the slowest rank's times, and the reported value counts the work
of all ranks over that time."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_max_over_ranks([1.0 + rank, 10.0 - rank, 3.5], "cpu")
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 3.5]
    # one rank: the values as they are
    assert bench.reduce_max_over_ranks([4.0, 5.0], "cpu") == [4.0, 5.0]
    # two replicas of 3 steps of 100 units in the slowest rank's 2 s
    assert bench.job_throughput(2, 3, 100, 2.0) == 300.0
