"""The multi-GPU path is replicas only: every rank solves its own problems
and bench.py combines the ranks' figures (slowest time, summed FLOPs).
This checks that combination with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, f = bench.combine_over_ranks(1.0 + rank, 10.0 * (rank + 1), torch.device("cpu"))
    out[rank] = (t, f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_times_take_the_max_and_flops_the_sum():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == (2.0, 30.0) and res[1] == (2.0, 30.0)


def test_single_process_is_identity():
    import bench
    assert bench.combine_over_ranks(3.5, 7.0, torch.device("cpu")) == (3.5, 7.0)
