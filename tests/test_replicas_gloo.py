"""The N > 1 path of bench.py ("replicas only": each rank integrates its own
replica, only the timing is reduced) on two CPU ranks over gloo."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = 0.010 * (rank + 1)             # rank 1 is the slowest
    slow = bench.slowest_rank(secs, torch.device("cpu"), dist)
    thr = bench.job_throughput(1_000_000, secs, torch.device("cpu"), world, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slow, thr))


def test_two_gloo_ranks_reduce_to_the_slowest_replica():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, thr in out:
        assert slow == pytest.approx(0.020)
        assert thr == pytest.approx(world * 1_000_000 / 0.020 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(0.5, torch.device("cpu")) == 0.5
    assert bench.job_throughput(2e9, 0.5, torch.device("cpu")) == pytest.approx(4.0)
