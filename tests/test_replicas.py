"""CPU test of the multi-process (replica) path of the benchmark: two gloo ranks on
127.0.0.1, each timing its own replica. The job's time is the slowest rank's and the
job's rate counts the work of every rank; a rank that fails makes the launch fail."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.env_rank()
    assert (r, w, lr) == (rank, world, rank)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    worst = bench.max_over_ranks(ms, dist)
    rate = bench.job_rate(w, 1000.0, worst)
    dist.barrier()
    out[rank] = (worst, rate)
    dist.destroy_process_group()


def test_two_gloo_replicas_time_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert out[0] == out[1] == (15.0, 2 * 1000.0 / 15e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 10.0, 2.0) == 5000.0
