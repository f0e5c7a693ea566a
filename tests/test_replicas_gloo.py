"""The bench's multi-GPU path is replicas only: each rank times its own loop,
the job time is the max over ranks and value = all ranks' iterations / that
time.  Checked here with two gloo ranks on the CPU (no GPU, no NCCL)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 2.0 + rank  # rank 1 is slower
    t = bench.aggregate_time(t_local, dist, torch.device("cpu"))
    out[rank] = bench.job_value(steps=100, world=world, t_max=t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    # t_max = 3.0 s, 2 ranks x 100 iterations
    assert out[0] == pytest.approx(200 / 3.0) and out[1] == pytest.approx(200 / 3.0)
