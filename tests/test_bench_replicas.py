"""The multi-GPU path of bench.py (replicas, one solve stream per rank) on CPU.

Two gloo ranks stand in for two GPUs: each reports its own elapsed time; the
job's value must be the total number of solves over the slowest rank's time,
identical on every rank.  No GPU is involved (the solves themselves are
single-GPU and independent; only this aggregation crosses ranks).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]                  # rank 1 is the slow one
    value, worst = bench.aggregate_ranks(elapsed, steps=5, dist=dist, device="cpu")
    q.put((rank, value, worst))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, worst in res:
        assert worst == 3.0
        assert value == pytest.approx(2 * 5 / 3.0)


def test_single_rank_aggregation_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, worst = bench.aggregate_ranks(2.5, steps=5)
    assert worst == 2.5 and value == pytest.approx(2.0)
