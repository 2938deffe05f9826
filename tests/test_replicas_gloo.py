"""The benchmark's multi-process logic on CPU ranks (gloo, world size 2): the
per-step time is the maximum over ranks, the same on every rank, and the
aggregate rate counts every rank's queries (replicas, weak scaling)."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(1.0 + rank * 0.5, world, torch.device("cpu"))
        dist.barrier()
        out[rank] = ms
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate():
    import bench
    world = 2
    port = 29500 + (os.getpid() % 1000)
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == 1.5
    assert bench.replicas_value(1000, world, 1.5) == pytest.approx(2 * 1000 / 1.5e-3)
    assert bench.max_over_ranks(2.5, 1, torch.device("cpu")) == 2.5
