#!/usr/bin/env python3
"""Benchmark of the nonlocal hydrodynamic FDTD solve on GB300.

One benchmark step is one whole solve of the workload through every step of
the method: voxelise the geometry, build the coefficient tables, advance all
time steps (fused H/E/P_CP/P_f update with CPML and TF/SF, running FP64 DFT on
the flux boxes), and reduce the cross sections.  The workload is the 224^3
Au-like GNOR sphere with a Lorentz pole (r = 10 nm, dx = 0.2 nm, 12-cell CPML,
8000 steps, 200 frequencies); its state (~9 GB) is far larger than L2, so no
explicit L2 flush is needed between steps.

  value  - Gcell-updates/s on the device (CUDA events around each solve, the
           state already resident in HBM; nlf_reset re-voxelises and clears it)
  e2e    - the same metric through the public API from scratch: context
           creation, host->device upload of the problem, the solve and the
           device->host read of the spectra, timed on the host
  roofline - the EM step (k_step with k_step_pml running concurrently on a
           second stream; the dominant work of a time step): algorithmic
           bytes per launch over its mean CUDA-event duration (events around
           each kernel of the last 64 time steps of each solve, replayed as
           one CUDA graph) against the measured HBM copy bandwidth; the
           material update and DFT kernels are reported beside it
  cpu_baseline - the FP64 CPU oracle on a bounded sample of the same workload
  serving - solves/s and p50/p99 latency of the seeded request stream's first
           requests, continuous batching against one grid at a time
  batched - the 64-instance batched configuration (uneven 40^3..128^3 grids,
           4000 time steps each) advanced together by nlf_batch_run, against
           the same solves run one grid per launch sequence (wall time)

`--impl reference` times the oracle alone (the reference arm).  With several
GPUs (torchrun) every rank runs its own independent replica ("replicas only":
the solve is not sharded), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "sphere_au_gnor_r10nm_224"
METRIC = "nonlocal FDTD Gcell-updates/s"
UNIT = "Gcell-updates/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = []
        mx = 0.0
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
            except ValueError:
                continue
            for nm, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(prob, steps, gpu_check=False):
    """Time the FP64 oracle on `steps` time steps of the workload (host cores).
    With gpu_check, also advance the same problem by the same steps on the GPU
    and return the relative L2 error of each vector field against the oracle."""
    import numpy as np
    import oracle
    oracle.build()
    s = oracle.Sim(prob)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    cells = prob["shape"][0] * prob["shape"][1] * prob["shape"][2]
    acc = None
    if gpu_check:
        from paper_2005_06997_gb300 import nlfdtd
        g = nlfdtd.Solver(prob)
        g.run(steps)
        g.sync()
        acc = {}
        for vec, comps in (("E", ("Ex", "Ey", "Ez")), ("H", ("Hx", "Hy", "Hz"))):
            num = den = 0.0
            for c in comps:
                ref = np.asarray(s.array(c), dtype=np.float64)
                got = g.field(c).astype(np.float64)
                num += float(np.sum((got - ref) ** 2))
                den += float(np.sum(ref ** 2))
            acc[vec] = math.sqrt(num / den) if den > 0 else math.sqrt(num)
        g.close()
    s.close()
    return cells * steps / dt / 1e9, dt, acc


def oracle_one_thread(steps):
    """The oracle on `steps` steps of the workload with one host thread (a
    separate process, since the OpenMP team size is fixed at first use)."""
    code = ("import sys, time, math; sys.path.insert(0, %r); import oracle; "
            "from paper_2005_06997_gb300 import workloads as W; p = W.CONFIGS[%r](); s = oracle.Sim(p); "
            "t = time.perf_counter(); s.step(%d); dt = time.perf_counter() - t; "
            "print(math.prod(p['shape']) * %d / dt / 1e9, dt)") % (ROOT, WORKLOAD, steps, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    v, dt = out.stdout.split()[-2:]
    return float(v), float(dt)


def replica_time_ms(local_ms, dist, device):
    """Replicas only: every rank solves its own grid; the job time is the
    slowest rank's (all ranks receive it)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, cell_updates_per_rank, job_ms):
    """Whole-job Gcell-updates/s: the cell updates of all ranks over the job time."""
    return world * cell_updates_per_rank / (job_ms * 1e-3) / 1e9


def run_reference(args, rank, world):
    from paper_2005_06997_gb300 import workloads as W
    prob = W.CONFIGS[WORKLOAD]()
    if rank != 0:
        return
    sample_steps = prob["monitors"]["K"]
    vals = []
    for _ in range(args.warmup):
        oracle_sample(prob, 2)
    t_all = 0.0
    for _ in range(args.steps):
        v, dt, _ = oracle_sample(prob, sample_steps)
        vals.append(v)
        t_all += dt
    value = args.steps * sample_steps * math.prod(prob["shape"]) / t_all / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": math.prod(prob["shape"]), "time_steps_per_step": sample_steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d time steps of the %s grid per step (FP64 oracle)" % (sample_steps, WORKLOAD)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, dist):
    import torch
    from paper_2005_06997_gb300 import nlfdtd
    from paper_2005_06997_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    prob = W.CONFIGS[WORKLOAD]()
    steps = prob["steps"]
    cells = math.prod(prob["shape"])
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    solver = nlfdtd.Solver(prob)
    solver.reset(sp)
    info = solver.info()
    step_bytes = info["step_bytes"]
    K = prob["monitors"]["K"]
    tail = 64          # single-step launches at the end of each solve, timed one by one

    def solve(record_kernel_times=None):
        solver.reset(sp)
        solver.run(steps - tail, sp)
        if record_kernel_times is not None:
            # the last steps with CUDA events around each kernel (one captured graph)
            record_kernel_times.append(solver.time_kernels(tail, sp))
        else:
            solver.run(tail, sp)
        return solver.spectra()

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = solver.launches
    kernel_ev = []
    times = []
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        spec = solve(kernel_ev)
        b.record(stream)
        times.append((a, b))
    t_stop.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    launches = solver.launches - launches0
    total_ms = replica_time_ms(t_start.elapsed_time(t_stop), dist, "cuda")
    n_timed = tail * len(kernel_ev)
    k_mean_ms = sum(t["step_ms"] for t in kernel_ev) / n_timed
    m_mean_ms = sum(t["metal_ms"] for t in kernel_ev) / n_timed
    d_mean_ms = sum(t["dft_ms"] for t in kernel_ev) / n_timed
    peak, peak_kind = peaks()
    step_kernel_bytes = info["step_kernel_bytes"]
    metal_kernel_bytes = info["metal_kernel_bytes"]
    achieved = step_kernel_bytes / (k_mean_ms * 1e-3) / 1e9
    value = replica_value(world, args.steps * steps * cells, total_ms)

    # end to end through the public API: create, upload, solve, read the spectra
    torch.cuda.synchronize()
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1, min(3, args.steps))):
        t0 = time.perf_counter()
        s2 = nlfdtd.Solver(prob)
        s2.run(steps, sp)
        sp2 = s2.spectra()
        t1 = time.perf_counter()
        inf2 = s2.info()
        h2d, d2h = inf2["h2d_bytes"], inf2["d2h_bytes"]
        s2.close()
        e2e_times.append(t1 - t0)
    e2e_val = steps * cells / statistics.mean(e2e_times) / 1e9 * world
    del solver

    serving = None
    if args.serving > 0:
        serving = run_serving(args.serving)
    batched = run_batched(args.batched) if args.batched > 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = prob["monitors"]["K"]
        v, dt, acc = oracle_sample(prob, sample, gpu_check=True)
        cpu = {"value": v, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
               "kind": "oracle", "sample": "%d time steps of the %s grid (FP64 oracle, %.1f s)" %
               (sample, WORKLOAD, dt),
               "gpu_rel_l2_vs_oracle": acc}
        try:
            v1, dt1 = oracle_one_thread(2)
            cpu["one_thread"] = {"value": v1, "sample": "2 time steps, one host thread (%.1f s)" % dt1}
        except Exception as e:              # report, do not fail the benchmark line
            cpu["one_thread"] = {"error": str(e)[:200]}

    if rank == 0:
        traffic = None
        tp = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
        if os.path.exists(tp):
            try:
                with open(tp) as f:
                    tr = json.load(f)
                if tr.get("workload") == WORKLOAD and tr.get("kernel_hash") == kernel_hash():
                    traffic = tr["bytes_per_launch"]
            except Exception:
                traffic = None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "time_steps_per_step": steps,
                       "grid": list(prob["shape"]), "dx_m": prob["dx"], "frequencies": len(prob["monitors"]["omega"]),
                       "l2": "state %.1f GB > 129 MB L2, no flush needed" % (info_bytes(prob) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "EM step: k_step + k_step_pml (concurrent), per time step",
                         "kernel_ms": k_mean_ms, "bytes_per_launch": step_kernel_bytes},
            "kernels_per_time_step": {
                "k_step": {"ms": k_mean_ms, "bytes": step_kernel_bytes,
                           "gbs": step_kernel_bytes / (k_mean_ms * 1e-3) / 1e9},
                "k_post": {"what": "material update and TF/SF corrections, one launch (bytes: material sites)",
                           "ms": m_mean_ms, "bytes": metal_kernel_bytes,
                           "gbs": metal_kernel_bytes / (m_mean_ms * 1e-3) / 1e9 if m_mean_ms > 0 else None},
                "dft": {"ms": d_mean_ms},
                "step_bytes": step_bytes},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "spectrum_peak_ev": float(prob["monitors"]["omega"][int(spec["ext"].argmax())] / W.EV_TO_RAD),
        }
        if serving is not None:
            line["serving"] = serving
        if batched is not None:
            line["batched"] = batched
        print(json.dumps(line), flush=True)


def run_serving(n):
    """The first n requests of the seeded Poisson stream (20 req/s; sphere /
    dimer / cube-with-tips solves on 48^3..320^3 grids, 2000..8000 steps, GNOR
    on or off) served by continuous batching with HBM-budget admission, and by
    the plain one-grid-at-a-time FIFO form; then the same requests arriving
    at 0.7 of the measured batched capacity, where latency is not queueing."""
    from paper_2005_06997_gb300 import serve
    from paper_2005_06997_gb300 import workloads as W
    reqs = W.serving_requests()[:n]
    out = {"requests": n, "rate_req_per_s": 20.0, "hbm_budget_gb": 200}
    _, sb = serve.Server(hbm_budget_bytes=200 << 30).run(reqs)
    _, sf = serve.serve_fifo(reqs)
    keys = ("solves_per_s", "p50_latency_s", "p99_latency_s", "gcell_updates_per_s", "wall_s")
    out["batched"] = {k: sb[k] for k in keys}
    out["fifo"] = {k: sf[k] for k in keys}
    # the same requests arriving at 0.7 of the batched capacity just measured
    # (the stated rate is ~10x what one GPU serves, so its latency is queueing)
    rate = 0.7 * sb["solves_per_s"]
    reqs07 = W.serving_requests(rate=rate)[:n]
    _, sb7 = serve.Server(hbm_budget_bytes=200 << 30).run(reqs07)
    _, sf7 = serve.serve_fifo(reqs07)
    out["load_0p7"] = {"rate_req_per_s": rate, "batched": {k: sb7[k] for k in keys},
                       "fifo": {k: sf7[k] for k in keys}}
    return out


def run_batched(n):
    """The batched configuration: n independent sphere / dimer solves on
    uneven grids (40^3..128^3, seeded), 4000 time steps each, advanced
    together by nlf_batch_run (one launch sequence per time step over all
    grids, replayed from captured CUDA graphs), against the same solves run
    one grid per launch sequence.  Wall time from the first launch to the
    last spectra, with a device synchronisation on both sides; each form is
    warmed up (plans, graphs, tile autotuning) and reset before it is timed."""
    import torch

    from paper_2005_06997_gb300 import nlfdtd
    from paper_2005_06997_gb300 import workloads as W
    probs = W.batched_instances(n=n)
    steps = int(probs[0]["steps"])
    cells = sum(math.prod(p["shape"]) for p in probs)
    solvers = [nlfdtd.Solver(p) for p in probs]
    try:
        def timed(go):
            for s in solvers:
                s.reset()
            torch.cuda.synchronize()
            t = time.perf_counter()
            go()
            for s in solvers:
                s.sync()
                s.spectra()
            torch.cuda.synchronize()
            return time.perf_counter() - t

        def batched(k):
            st = nlfdtd.batch_run(solvers, [k] * n)
            if any(st):
                raise RuntimeError("batched solve status %s" % st)

        def alone(k):
            for s in solvers:
                s.run(k)

        timed(lambda: batched(512))
        t_b = timed(lambda: batched(steps))
        timed(lambda: alone(512))
        t_a = timed(lambda: alone(steps))
    finally:
        for s in solvers:
            s.close()
    upd = float(cells) * steps

    def line(t):
        return {"wall_s": t, "gcell_updates_per_s": upd / t / 1e9, "solves_per_s": n / t}

    return {"instances": n, "time_steps": steps, "cells": cells, "cell_updates": upd,
            "batched": line(t_b), "one_grid_per_launch": line(t_a)}


def info_bytes(prob):
    from paper_2005_06997_gb300 import nlfdtd
    s = nlfdtd.Solver(prob)
    b = s.state_bytes()
    s.close()
    return b


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for fn in ("step.cu", "nlf_internal.h"):
        with open(os.path.join(ROOT, "paper_2005_06997_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=48, help="requests of the serving stream to run (0: skip)")
    ap.add_argument("--batched", type=int, default=64, help="instances of the batched configuration (0: skip)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist_mod.init_process_group(backend=backend)
        dist = dist_mod
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        from paper_2005_06997_gb300 import build
        if rank == 0:
            build.build()
        if dist is not None:
            dist.barrier()
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
