"""The multi-GPU form is replicas only: each rank solves its own grid and the
job time is the slowest rank's.  The aggregation bench.py uses, checked with
two gloo ranks on CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [120.0, 250.0][rank]                 # rank 1 is the slower replica
        job = bench.replica_time_ms(local, dist, "cpu")
        out[rank] = (job, bench.replica_value(world, 1.0e9, job))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    port = 29000 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        job, value = res[r]
        assert job == 250.0
        assert value == pytest.approx(2 * 1.0e9 / 0.25 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_time_ms(42.0, None, "cpu") == 42.0
    assert bench.replica_value(1, 5.0e9, 1000.0) == pytest.approx(5.0)
