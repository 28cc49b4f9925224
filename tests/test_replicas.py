"""The multi-GPU path of the benchmark is "replicas only": N independent
copies of the solve, no data-path collective.  Its host logic -- the job's
time as the slowest rank's (a MAX all-reduce) and the whole-job throughput
N x units / that time -- runs here on two CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 100 units
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        out[rank] = (t, bench.replica_rate(100.0, world, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert dict(out) == {0: (2.0, 100.0), 1: (2.0, 100.0)}


def test_single_rank_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_rate(262144 * 20, 1, 0.025) == 262144 * 20 / 0.025
