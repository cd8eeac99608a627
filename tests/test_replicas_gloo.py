"""Multi-rank timing of bench.py's replica mode on CPU (gloo, world size 2).

The query has no exchange step, so N GPUs run N independent replicas; the
whole-job rate is the units all ranks processed divided by the slowest rank's
time.  This checks that reduction with two real processes.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(10.0 * (rank + 1), 1000, world, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_aggregate_ranks_two_processes():
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
    for rank, ms, value in res:
        assert ms == 20.0                        # slowest rank
        assert value == pytest.approx(2 * 1000 / 0.020)


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(5.0, 100, 1, "cpu") == (5.0, pytest.approx(100 / 0.005))
