"""The multi-rank (replica) reduction of bench.py on two CPU ranks (gloo):
the step time is the slowest rank's, the ray count the sum of all ranks'."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx, sm = bench.reduce_over_ranks([1.5 + rank, 10.0 * (rank + 1)], [100.0 * (rank + 1), 7.0], "cpu")
    out[rank] = (mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        mx, sm = out[r]
        assert mx == [2.5, 20.0]
        assert sm == [300.0, 14.0]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([3.0], [4.0], "cpu") == ([3.0], [4.0])
