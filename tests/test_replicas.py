"""Host logic of bench.py.  The multi-GPU form is replicas only: each rank
solves its own grid and the job time is the slowest rank's (the aggregation
checked with two gloo ranks on CPU); the serving section's child process
reports its failures in the section."""
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


def test_serving_child_failure_is_reported_in_its_section(monkeypatch):
    """The benchmark's serving section runs in a child process: a child that
    fails or runs out of time leaves a section that says so, and a child
    that succeeds hands over its JSON line."""
    import subprocess
    import types
    sys.path.insert(0, ROOT)
    import bench

    def timeout(cmd, **kw):
        raise subprocess.TimeoutExpired(cmd, kw.get("timeout"))

    monkeypatch.setattr(bench.subprocess, "run", timeout)
    out = bench.run_serving_child(16, timeout_s=5)
    assert out == {"requests": 16, "error": "no result within 5 s"}

    def crash(cmd, **kw):
        assert "--serving-child" in cmd and "16" in cmd
        return types.SimpleNamespace(returncode=1, stdout="", stderr="line one\nRuntimeError: no device\n")

    monkeypatch.setattr(bench.subprocess, "run", crash)
    out = bench.run_serving_child(16)
    assert out["requests"] == 16 and out["error"] == "exit 1: RuntimeError: no device"

    def ok(cmd, **kw):
        return types.SimpleNamespace(returncode=0, stdout='note\n{"requests": 16, "batched": {}}\n', stderr="")

    monkeypatch.setattr(bench.subprocess, "run", ok)
    assert bench.run_serving_child(16) == {"requests": 16, "batched": {}}
