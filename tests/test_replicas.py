"""Multi-GPU form of the bench: replicas with no data-path collective (the path does not shard).

Two gloo ranks on the CPU stand in for two GPUs: each reports its own time, the job's time is the
slowest rank's, and the job's value counts the points of every rank.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, device="cpu")
    out[rank] = (ms, bench.job_value(world, 1000, 10, ms))
    dist.destroy_process_group()


def test_replica_timing_is_the_slowest_rank_and_value_counts_all_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()     # no fork of this (threaded) test process
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 150.0
    assert abs(out[0][1] - 2 * 1000 * 10 / 0.150 / 1e9) < 1e-15
