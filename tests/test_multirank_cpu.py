"""The replicas-only multi-GPU path of bench.py: each rank times its own solves, the job takes the
slowest rank's time and counts every rank's solves. Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = [2.0, 3.5][rank]
    slowest = bench.max_over_ranks(local_seconds)
    out[rank] = (slowest, bench.whole_job_rate(10, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1] == (3.5, 20 / 3.5)


def test_single_process_without_group():
    import bench

    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_rate(7, 1, 2.0) == 3.5
