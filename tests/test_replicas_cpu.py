"""Replica host logic of bench.py at world size 2 with the gloo backend (no GPU).

N replicas run independent fits; the job's throughput is all iterations over the slowest rank's time
(max over ranks), the only collective being that one scalar all-reduce.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, ms = bench.replica_throughput(local_ms[rank], steps, world, dist, "cpu")
        out[rank] = (value, ms)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    world, steps = 2, 100
    local_ms = [50.0, 80.0]          # rank 1 is slower
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, local_ms, steps, out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        value, ms = out[rank]
        assert ms == pytest.approx(80.0 / steps)
        assert value == pytest.approx(world * steps / 0.080)


def test_single_process_needs_no_collective():
    import bench
    value, ms = bench.replica_throughput(40.0, 10, 1, None, None)
    assert ms == pytest.approx(4.0)
    assert value == pytest.approx(10 / 0.040)
