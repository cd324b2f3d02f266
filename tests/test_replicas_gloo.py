"""The benchmark's multi-replica host logic on CPU: two gloo ranks, each with
its own time; every rank sees the slowest time, and the job rate counts the
units of all ranks over it (replicas only: no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = bench.max_over_ranks(times[rank], world)
    out[rank] = (t, bench.job_rate(1000, 10, t, world))
    dist.destroy_process_group()


def test_two_rank_max_time_and_job_rate():
    world, port = 2, _free_port()
    times = [0.5, 2.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, times, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1] == (2.0, 2 * 1000 * 10 / 2.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_rate(60_000_000, 20, 0.5, 1) == pytest.approx(2.4e9)
