"""Multi-process (world size 2, gloo on CPU) path of bench.py's timing aggregation.

On N GPUs every rank solves its own copy of the workload (independent
instances, no collective on the data path); the only exchange is the max over
ranks of the timed region, from which the whole-job throughput is formed.
"""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        m = bench.max_over_ranks(times[rank], dist)
        out[rank] = m
        out[world + rank] = bench.job_throughput(1000.0, world, 4, m)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo_world2():
    world, port = 2, _free_port()
    times = [12.5, 40.0]                 # ms of the timed region on each rank
    out = torch.zeros(2 * world, dtype=torch.float64).share_memory_()
    mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
    assert out[0].item() == out[1].item() == 40.0
    # 2 ranks x 1000 units x 4 steps over the slowest rank's 40 ms
    assert out[2].item() == pytest.approx(2 * 1000 * 4 / 0.040)
    assert out[3].item() == out[2].item()


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_throughput(10.0, 1, 2, 4.0) == pytest.approx(5000.0)
