"""The multi-GPU path is replicas only (the solve does not shard): each rank solves its own
copy of the workload and bench.py reports all ranks' solves over the slowest rank's time.
This checks that aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [2.0, 3.0][rank]      # seconds of the rank's timed region
    n_local = [3, 3][rank]          # solves the rank completed
    value, tmax, n = bench.aggregate(t_local, n_local, dist, torch.device("cpu"))
    dist.barrier()
    out[rank] = (value, tmax, n)
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of this (multi-threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, tmax, n = out[r]
        assert tmax == 3.0 and n == 6
        assert abs(value - 2.0) < 1e-12
