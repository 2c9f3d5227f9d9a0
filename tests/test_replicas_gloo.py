"""Multi-GPU path of bench.py (independent replicas, no data-path collective) on CPU ranks.

Two gloo ranks stand in for two GPUs: each reports its own timed-region length, the job's
time is the maximum over ranks, and the value counts the units of every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, "cpu")
        out[rank] = (ms, bench.replica_throughput(10, 5, ms, ws))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mgr = mp.Manager()
    out = mgr.dict()
    port = free_port()
    mp.spawn(rank_main, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        ms, rate = out[rank]
        assert ms == pytest.approx(150.0)
        assert rate == pytest.approx(2 * 10 * 5 / 0.150)


def test_single_process_needs_no_collective():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.replica_throughput(7, 3, 1000.0, 1) == pytest.approx(21.0)
