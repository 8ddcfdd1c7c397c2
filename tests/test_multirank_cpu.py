"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only -- the
solver path has no data-path collective; only the timing aggregation talks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, it = bench.aggregate_ranks(dev_s=1.0 + rank, iters=100 * (rank + 1), dist=dist, device="cpu")
    out[rank] = (t, it)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_max_time_sum_iterations():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == (2.0, 300.0) and out[1] == (2.0, 300.0)


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_ranks(1.5, 7) == (1.5, 7.0)
