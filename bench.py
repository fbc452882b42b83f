#!/usr/bin/env python3
"""Benchmark of the nonlocal hydrodynamic FDTD solve on GB300.

One benchmark step is one whole solve of the workload through every step of
the method: voxelise the geometry, build the coefficient tables, advance all
time steps (fused H/E/P_CP/P_f update with CPML and TF/SF, running FP64 DFT on
the flux boxes), and reduce the cross sections.  The headline workload is the
largest single-GPU configuration: the 512^3 Au-like GNOR cube with six
rounded pyramidal tips (60 nm cube, 3 nm apex radius, dx = 0.25 nm, 12-cell
CPML, 10000 time steps, 1-5 eV, 200 frequencies; ~37 GB of state, far larger
than L2, so no explicit L2 flush is needed between steps).  The 224^3 Au-like
GNOR sphere with a Lorentz pole (8000 steps) is reported beside it under
"workloads".

  value  - Gcell-updates/s on the device (CUDA events around the timed solves,
           the state already resident in HBM; nlf_reset re-voxelises and clears it)
  e2e    - the same metric through the public API from host inputs: context
           creation, host->device upload of the problem, the solve and the
           device->host read of the spectra, timed on the host
  roofline - the EM step (k_step with k_step_pml running concurrently on a
           second stream; the dominant work of a time step): algorithmic
           bytes per launch over its mean CUDA-event duration (events around
           each kernel of the last 64 time steps of each solve, replayed as
           one CUDA graph) against the measured HBM copy bandwidth; the
           material update and DFT kernels are reported beside it
  whole_step - the whole solve's time per time step against the hot-path
           byte count of one time step (fields, hydrodynamic state, CPML,
           material ids, running DFT)
  cpu_baseline - the FP64 CPU oracle on a bounded sample of the same workload
  serving - solves/s and p50/p99 latency of the seeded request stream's
           first N requests (--serving N; default 128 on one GPU, none under
           torchrun), continuous batching against one grid at a time, at the
           stated 20 req/s and at 0.7 of the plain form's capacity; run in a
           child process after the other sections (a failure there is
           reported in the section and leaves the line intact); the whole
           256-request stream (--serving 256) takes about five and a half
           minutes
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

HEADLINE = "cube_tips_au_gnor_512"
SECOND = "sphere_au_gnor_r10nm_224"
HEADLINE_SEGMENT = 1000       # time steps per benchmark step (a tenth of the headline solve)
REF_SAMPLE_STEPS = 1          # oracle time steps per reference-arm step
CPU_SAMPLE_STEPS = 8          # oracle time steps of the cpu_baseline sample
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
    s.step(1)                     # first touch of the oracle's arrays, untimed
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    cells = prob["shape"][0] * prob["shape"][1] * prob["shape"][2]
    acc = None
    if gpu_check:
        from paper_2005_06997_gb300 import nlfdtd
        g = nlfdtd.Solver(prob)
        g.run(steps + 1)
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


def host_mem_available():
    """Bytes of host memory available now (Linux), or None."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        return None
    return None


def oracle_bytes(prob):
    """Host memory the FP64 oracle holds for a problem: full-grid FP64 arrays
    (E with two histories, H, P_f with two histories, two grad-div histories
    and the current one, CPML psi for every component and axis, the poles'
    three generations) plus the DFT accumulators."""
    cells = math.prod(prob["shape"])
    poles = max([len(m.get("poles", [])) for m in prob.get("materials", [])] + [0])
    arrays = 9 + 3 + 9 + 9 + 18 + 9 * poles
    nrec = 0
    mo = prob.get("monitors")
    if mo is not None:
        for lo, hi in ((mo["abs_lo"], mo["abs_hi"]), (mo["sca_lo"], mo["sca_hi"])):
            e = [h - l + 1 for l, h in zip(lo, hi)]
            nrec += 4 * (e[0] * e[1] + e[1] * e[2] + e[0] * e[2])
        nrec = nrec * len(mo["omega"]) * 32
    return arrays * 8 * cells + nrec


def baseline_workload(name):
    """The workload the oracle can be timed on here: `name` itself when its
    arrays fit the host's available memory (with a 25 % margin), else None."""
    from paper_2005_06997_gb300 import workloads as W
    prob = W.CONFIGS[name]()
    avail = host_mem_available()
    need = oracle_bytes(prob)
    if avail is not None and need * 1.25 > avail:
        return None, need, avail
    return prob, need, avail


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, created once for
    the headline workload (its set-up untimed); each benchmark step advances
    it REF_SAMPLE_STEPS time steps."""
    if rank != 0:
        return
    import oracle
    prob, need, avail = baseline_workload(HEADLINE)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    if prob is None:
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle of %s needs %.0f GB of host memory, "
                          "%.0f GB available" % (HEADLINE, need / 1e9, (avail or 0) / 1e9)}), flush=True)
        return
    oracle.build()
    sim = oracle.Sim(prob)
    for _ in range(args.warmup):
        sim.step(REF_SAMPLE_STEPS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step(REF_SAMPLE_STEPS)
    t_all = time.perf_counter() - t0
    sim.close()
    value = args.steps * REF_SAMPLE_STEPS * math.prod(prob["shape"]) / t_all / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE, "cells": math.prod(prob["shape"]), "time_steps_per_step": REF_SAMPLE_STEPS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d time step(s) of the %s grid per step (FP64 oracle, set up once, untimed)"
                         % (REF_SAMPLE_STEPS, HEADLINE)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def survey_step_bytes(info, prob):
    """Algorithmic HBM bytes of one whole time step by the hot-path byte
    count: 48 per cell (E and H read and written once, FP32), 8 (2 + g +
    2 poles) per plasmonic E-site (P_f, a_f, the GNOR history, P_CP and a_CP
    read and written), 32 per CPML slab cell and axis (two psi_E and two psi_H
    read and written), 1 per bounding-box site (the material id), and the
    running DFT: 12 bytes per record every K steps (E, H samples) and 32 bytes
    per record and frequency per flush of B samples (FP64 accumulators read
    and written)."""
    mo = prob.get("monitors")
    dft = 0.0
    if mo is not None:
        nf = len(mo["omega"])
        K = mo.get("K", 16)
        B = 32
        nrec = info["dft_records"] + 1
        dft = 12.0 * nrec / K + 32.0 * nrec * nf / (B * K)
    g = 1 if info["gnor"] else 0
    metal = 8.0 * (2 + g + 2 * info["n_poles"]) * info["metal_sites"] + 3.0 * info["bbox_cells"]
    return 48.0 * info["cells"] + 32.0 * info["pml_slab_cells"] + metal + dft


def measure(name, n_steps, n_warmup, dist, dev, stream, e2e_reps, seg=None, tail=64):
    """Device-timed solves of workload `name` (state resident in HBM).  One
    benchmark step is a segment of `seg` time steps (default: the whole
    solve); a solve is steps / seg consecutive segments, the first one
    starting with nlf_reset (clear, re-voxelise, upload the tables) and the
    last one ending with the cross sections.  The timed region starts with a
    fresh solve.  CUDA events around each kernel of the last `tail` time
    steps of every solve give the per-kernel figures; the end-to-end rate is
    taken through the C ABI from host inputs."""
    import torch
    from paper_2005_06997_gb300 import nlfdtd
    from paper_2005_06997_gb300 import workloads as W

    prob = W.CONFIGS[name]()
    steps = prob["steps"]
    seg = steps if seg is None else seg
    assert steps % seg == 0 and seg > tail
    per_solve = steps // seg
    cells = math.prod(prob["shape"])
    sp = stream.cuda_stream
    solver = nlfdtd.Solver(prob)
    solver.reset(sp)
    info = solver.info()
    out = {}

    def segment(pos, record_kernel_times=None):
        if pos == 0:
            solver.reset(sp)
        if pos == per_solve - 1:
            if record_kernel_times is not None:
                solver.run(seg - tail, sp)
                record_kernel_times.append(solver.time_kernels(tail, sp))
            else:
                solver.run(seg, sp)
            out["spec"] = solver.spectra()
        else:
            solver.run(seg, sp)

    for w in range(n_warmup):
        segment(w % per_solve)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = solver.launches
    kernel_ev = []
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for w in range(n_steps):
        segment(w % per_solve, kernel_ev)
    t_stop.record(stream)
    launches = solver.launches - launches0
    # finish the solve in progress (untimed) for the kernel figures and the
    # comparison with the oracle's stored full-length run
    w = n_steps
    while w % per_solve:
        segment(w % per_solve, kernel_ev)
        w += 1
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    world = dist.get_world_size() if dist is not None else 1
    total_ms = replica_time_ms(t_start.elapsed_time(t_stop), dist, "cuda")
    n_timed = tail * len(kernel_ev)
    k_ms = sum(t["step_ms"] for t in kernel_ev) / n_timed
    m_ms = sum(t["metal_ms"] for t in kernel_ev) / n_timed
    d_ms = sum(t["dft_ms"] for t in kernel_ev) / n_timed
    golden = golden_errors(solver, name, out["spec"])
    peak, peak_kind = peaks()
    kb = info["step_kernel_bytes"]
    mb = info["metal_kernel_bytes"]
    sb = survey_step_bytes(info, prob)
    ms_per_time_step = total_ms / (n_steps * seg)
    value = replica_value(world, n_steps * seg * cells, total_ms)
    solver.close()

    # end to end through the public API from host inputs: create, upload and
    # voxelise, solve, read the spectra back; host clock around each
    torch.cuda.synchronize()
    e2e_times = []
    h2d = d2h = 0
    for _ in range(e2e_reps):
        t0 = time.perf_counter()
        s2 = nlfdtd.Solver(prob)
        s2.run(steps, sp)
        s2.spectra()
        t1 = time.perf_counter()
        inf2 = s2.info()
        h2d, d2h = inf2["h2d_bytes"], inf2["d2h_bytes"]
        s2.close()
        e2e_times.append(t1 - t0)
    e2e_val = steps * cells / statistics.mean(e2e_times) / 1e9 * world

    traffic = None
    tp = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if os.path.exists(tp):
        try:
            with open(tp) as f:
                tr = json.load(f)
            ent = tr.get(name) if isinstance(tr, dict) else None
            if ent and ent.get("kernel_hash") == kernel_hash():
                traffic = ent["bytes_per_launch"]
        except Exception:
            traffic = None
    ext = out["spec"]["ext"]
    return {
        "workload": name, "value": value, "ms_per_step": total_ms / n_steps, "steps": n_steps,
        "warmup": n_warmup, "cells": cells, "time_steps_per_step": seg, "time_steps_per_solve": steps,
        "launches": launches,
        "grid": list(prob["shape"]), "dx_m": prob["dx"],
        "frequencies": len(prob["monitors"]["omega"]), "state_gb": info_bytes(prob) / 1e9,
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": kb / (k_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": kb / (k_ms * 1e-3) / 1e9 / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "EM step: k_step and k_step_pml (concurrent), then k_step_metal where the "
                               "material update is fused into the z march; per time step",
                     "kernel_ms": k_ms, "bytes_per_launch": kb},
        "whole_step": {"ms": ms_per_time_step, "bytes": sb,
                       "gbs": sb / (ms_per_time_step * 1e-3) / 1e9,
                       "frac": sb / (ms_per_time_step * 1e-3) / 1e9 / peak,
                       "what": "whole solve time per time step (reset, voxelise, every step, DFT, spectra) "
                               "against the hot-path byte count of one time step"},
        "kernels_per_time_step": {
            "em_step": {"ms": k_ms, "bytes": kb, "gbs": kb / (k_ms * 1e-3) / 1e9},
            "k_post": {"what": "material update and TF/SF corrections (bytes: material sites)",
                       "ms": m_ms, "bytes": mb, "gbs": mb / (m_ms * 1e-3) / 1e9 if m_ms > 0 else None},
            "dft": {"ms": d_ms}},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "spectrum_peak_ev": float(prob["monitors"]["omega"][int(ext.argmax())] / W.EV_TO_RAD),
        "error_vs_oracle": golden,
    }


def golden_errors(solver, name, spec):
    """Errors of a finished solve against the FP64 oracle's full-length run
    of the same problem (tests/golden/full_run_<name>.npz, written by
    tests/golden/make_full_run_golden.py): relative L2 of each vector field
    over the stored sample sites, relative error of each field's norm, the
    largest error of sigma_ext where I >= 1e-3 max I relative to its largest
    magnitude there, and the frequency index of the extinction maximum (GPU,
    oracle)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "full_run_%s.npz" % name)
    if not os.path.exists(path):
        return None
    g = np.load(path)
    out = {"golden": os.path.relpath(path, ROOT)}
    for vec in ("E", "H", "P"):
        num = den = 0.0
        n_got = n_ref = 0.0
        for c in "xyz":
            f = vec + c
            a = solver.field(f).astype(np.float64).reshape(-1)
            ref = g["val_" + f]
            num += float(np.sum((a[g["idx_" + f]] - ref) ** 2))
            den += float(np.sum(ref ** 2))
            n_got += float(np.sum(a * a))
            n_ref += float(g["sumsq_" + f])
        out["rel_l2_samples_" + vec] = math.sqrt(num / den) if den > 0 else None
        out["rel_norm_" + vec] = abs(math.sqrt(n_got) - math.sqrt(n_ref)) / math.sqrt(n_ref) if n_ref > 0 else None
    inc = g["inc"]
    m = inc >= 1e-3 * inc.max()
    out["sigma_ext_rel"] = float(np.max(np.abs(spec["ext"][m] - g["ext"][m])) / np.max(np.abs(g["ext"][m])))
    i_ref, i_got = int(np.argmax(g["ext"])), int(np.argmax(spec["ext"]))
    out["peak_index"] = [i_got, i_ref]
    return out


def run_ours(args, rank, world, dist):
    import torch

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    head = measure(HEADLINE, args.steps, args.warmup, dist, dev, stream, e2e_reps=1, seg=HEADLINE_SEGMENT)
    second = None
    if not args.headline_only:
        second = measure(SECOND, max(args.steps, 5), max(args.warmup, 3), dist, dev, stream, e2e_reps=3)
    batched = run_batched(args.batched) if args.batched > 0 else None
    n_serve = args.serving if args.serving >= 0 else (128 if world == 1 else 0)
    serving = None
    if n_serve > 0 and rank == 0:
        # the child gets the device memory this process no longer needs
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        serving = run_serving_child(n_serve)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        prob, need, avail = baseline_workload(HEADLINE)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        if prob is None:
            cpu = {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "not run: the FP64 oracle of %s needs %.0f GB of host memory, %.0f GB available"
                   % (HEADLINE, need / 1e9, (avail or 0) / 1e9)}
        else:
            v, dt, acc = oracle_sample(prob, CPU_SAMPLE_STEPS, gpu_check=True)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d time steps of the %s grid (FP64 oracle, %.1f s after its set-up)" %
                   (CPU_SAMPLE_STEPS, HEADLINE, dt),
                   "gpu_rel_l2_vs_oracle": acc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": HEADLINE, "cells": head["cells"], "time_steps_per_step": head["time_steps_per_step"],
                       "time_steps_per_solve": head["time_steps_per_solve"],
                       "step": "a segment of %d time steps; a solve is %d segments, the first re-voxelising "
                               "and clearing the state, the last reducing the cross sections"
                       % (head["time_steps_per_step"], head["time_steps_per_solve"] // head["time_steps_per_step"]),
                       "grid": head["grid"], "dx_m": head["dx_m"], "frequencies": head["frequencies"],
                       "l2": "state %.1f GB > 129 MB L2, no flush needed" % head["state_gb"],
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": head["roofline"],
            "whole_step": head["whole_step"],
            "kernels_per_time_step": head["kernels_per_time_step"],
            "e2e": head["e2e"],
            "gpu_launches": head["launches"],
            "clocks": head["clocks"],
            "cpu_baseline": cpu,
            "spectrum_peak_ev": head["spectrum_peak_ev"],
        }
        if second is not None:
            line["workloads"] = {SECOND: second}
        if serving is not None:
            line["serving"] = serving
        if batched is not None:
            line["batched"] = batched
        print(json.dumps(line), flush=True)


def run_serving(n):
    """The seeded request stream's first n requests (Poisson, 20 req/s;
    sphere / dimer / cube-with-tips solves on 48^3..231^3 grids, 2000..8000
    steps, GNOR on or off) served by the continuous-batching server (HBM
    budget admission, size-aware periods) and by the plain one-grid-at-a-time
    FIFO form; then the same requests arriving at 0.7 of the measured
    FIFO capacity, where latency is not queueing."""
    from paper_2005_06997_gb300 import serve
    from paper_2005_06997_gb300 import workloads as W
    reqs = W.serving_requests()[:n]
    out = {"requests": n, "rate_req_per_s": 20.0, "hbm_budget_gb": 200}
    keys = ("solves", "solves_per_s", "p50_latency_s", "p99_latency_s", "gcell_updates_per_s", "wall_s")
    _, sb = serve.Server(hbm_budget_bytes=200 << 30).run(reqs)
    _, sf = serve.serve_fifo(reqs)
    out["batched"] = {k: sb[k] for k in keys}
    out["fifo"] = {k: sf[k] for k in keys}
    # the same requests arriving at 0.7 of the plain form's capacity (the
    # stated rate is above what one GPU serves, so its latency is queueing)
    rate = 0.7 * sf["solves_per_s"]
    reqs07 = W.serving_requests(rate=rate)[:n]
    _, sb7 = serve.Server(hbm_budget_bytes=200 << 30).run(reqs07)
    _, sf7 = serve.serve_fifo(reqs07)
    out["load_0p7"] = {"rate_req_per_s": rate, "of": "fifo capacity", "batched": {k: sb7[k] for k in keys},
                       "fifo": {k: sf7[k] for k in keys}}
    return out


def run_serving_child(n, timeout_s=900):
    """run_serving(n) in a child process: its section of the line, or the
    reason it has none."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serving-child", str(n)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"requests": n, "error": "no result within %d s" % timeout_s}
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        tail = (r.stderr.strip().splitlines() or ["no output"])[-1]
        return {"requests": n, "error": "exit %d: %s" % (r.returncode, tail[:300])}
    return json.loads(lines[-1])


def run_batched(n):
    """The batched configuration: n independent sphere / dimer solves on
    uneven grids (40^3..128^3, seeded), 4000 time steps each, advanced
    together by nlf_batch_run (one launch sequence per time step over all
    grids, replayed from captured CUDA graphs), against the same solves run
    one grid per launch sequence.  Wall time from the first launch to the
    last spectra, with a device synchronisation on both sides; each form is
    warmed up and reset before it is timed: four DFT periods, so that the
    batched form has tuned its z chunk (three periods) and captured its
    plan's graph (the fourth), and the single grids have captured theirs."""
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

        warm = 4 * int(probs[0]["monitors"]["K"]) * 32       # a DFT period is K B steps (B = 32 here)
        timed(lambda: batched(warm))
        t_b = timed(lambda: batched(steps))
        timed(lambda: alone(warm))
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
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="skip the 224^3 section")
    ap.add_argument("--serving", type=int, default=-1,
                    help="requests of the serving stream to run (0: skip; default 128 on one GPU, 0 under torchrun)")
    ap.add_argument("--serving-child", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--batched", type=int, default=64, help="instances of the batched configuration (0: skip)")
    args = ap.parse_args()
    if args.serving_child > 0:
        # the serving section's child process (the library is already built)
        print(json.dumps(run_serving(args.serving_child)), flush=True)
        return
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
