"""Continuous-batching solve server over the C ABI (torch for memory and streams).

Requests (problem dicts with an ``arrival_s`` time) arrive on a clock.  The
server admits waiting requests first in, first out, while their state fits
the HBM budget and the batch has a free slot: each admitted request gets a
torch device buffer bound with ``nlf_bind_state`` and its state stays on the
device until it finishes.  All admitted requests advance together, one DFT
period (K * B time steps) per ``nlf_batch_run`` call, so requests that arrive
while others are running join at the next period boundary; finished requests
are retired there, their spectra copied out and their memory returned.

``serve_fifo`` is the plain form for comparison: one request at a time, in
arrival order, one grid per launch sequence.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import nlfdtd


class _Active:
    __slots__ = ("req", "solver", "buf", "remaining", "admit_s")

    def __init__(self, req, solver, buf, admit_s):
        self.req = req
        self.solver = solver
        self.buf = buf
        self.remaining = int(req["steps"])
        self.admit_s = admit_s


def _percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def summarise(results, wall_s):
    lat = [r["latency_s"] for r in results]
    work = sum(r["cell_updates"] for r in results)
    return {"solves": len(results), "wall_s": wall_s, "solves_per_s": len(results) / wall_s if wall_s > 0 else None,
            "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
            "gcell_updates_per_s": work / wall_s / 1e9 if wall_s > 0 else None}


class Server:
    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, stream=None):
        import torch
        nlfdtd.require_gpu()
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.used = 0
        self.launches = 0

    def _admit(self, req, now):
        s = nlfdtd.Solver(req, block_b=SERVE_B)
        nb = s.state_bytes()
        buf = self.torch.empty(nb + 256, dtype=self.torch.uint8, device="cuda")
        ptr = (buf.data_ptr() + 255) // 256 * 256
        s.bind_state(ptr, nb)
        s.reset(self.stream.cuda_stream)
        self.used += nb
        return _Active(req, s, buf, now)

    def _admit_waiting(self, waiting, active, sizes, now):
        """Admit waiting requests, first in first out, by HBM budget and slots."""
        while waiting and len(active) < self.max_active:
            req = waiting[0]
            key = id(req)
            if key not in sizes:
                probe = nlfdtd.Solver(req, block_b=SERVE_B)
                sizes[key] = probe.state_bytes()
                probe.close()
            if self.used + sizes[key] > self.budget and active:
                break
            waiting.popleft()
            active.append(self._admit(req, now))

    def run(self, requests, clock=time.perf_counter):
        """Serve `requests` (sorted by arrival_s); returns (results, summary).

        Each loop iteration enqueues one DFT period of the running batch, then
        admits the requests that arrived meanwhile on the host while the GPU
        works (their initialisation is queued behind the period on the same
        stream), then waits and retires the finished requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival_s"]))
        waiting = collections.deque()
        active = []
        results = []
        t0 = clock()
        sizes = {}
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0]["arrival_s"] <= now:
                waiting.append(pending.popleft())
            if not active:
                self._admit_waiting(waiting, active, sizes, now)
                if not active:
                    if pending:
                        time.sleep(max(0.0, min(0.05, pending[0]["arrival_s"] - (clock() - t0))))
                    continue
            U = _period(active[0])
            steps = [min(U, a.remaining) for a in active]
            running = list(active)
            before = sum(a.solver.launches for a in running)
            status = nlfdtd.batch_run([a.solver for a in running], steps, self.stream.cuda_stream)
            # host work while the GPU runs the period: admit new arrivals
            now = clock() - t0
            while pending and pending[0]["arrival_s"] <= now:
                waiting.append(pending.popleft())
            self._admit_waiting(waiting, active, sizes, now)
            self.stream.synchronize()
            self.launches += sum(a.solver.launches for a in running) - before
            now = clock() - t0
            done = set()
            for a, n, st in zip(running, steps, status):
                a.remaining -= n
                if st != 0 or a.remaining <= 0:
                    res = {"name": a.req.get("name"), "arrival_s": a.req["arrival_s"], "admit_s": a.admit_s,
                           "finish_s": now, "latency_s": now - a.req["arrival_s"], "status": int(st),
                           "cell_updates": float(np.prod(a.req["shape"])) * int(a.req["steps"])}
                    if st == 0:
                        res["spectra"] = a.solver.spectra()
                    results.append(res)
                    self.used -= a.solver.state_bytes()
                    a.solver.close()
                    a.buf = None
                    done.add(id(a))
            active = [a for a in active if id(a) not in done]
        wall = clock() - t0
        return results, summarise(results, wall)


# Samples buffered per DFT flush for served requests: a batched segment is one
# DFT period (K * SERVE_B steps), so this sets how often finished requests
# leave and new ones join.
SERVE_B = 16


def _period(a):
    """Time steps of one DFT period of an active request (the batching unit)."""
    mon = a.req.get("monitors")
    K = mon.get("K", 16) if mon else 1
    kb = K * SERVE_B
    return kb if kb % 2 == 0 else 2 * kb


def serve_fifo(requests, stream=None, clock=time.perf_counter):
    """One request at a time in arrival order (the plain one-grid-per-launch form)."""
    import torch
    nlfdtd.require_gpu()
    stream = stream if stream is not None else torch.cuda.Stream()
    results = []
    t0 = clock()
    launches = 0
    for req in sorted(requests, key=lambda r: r["arrival_s"]):
        now = clock() - t0
        if req["arrival_s"] > now:
            time.sleep(req["arrival_s"] - now)
        start = clock() - t0
        s = nlfdtd.Solver(req)
        s.run(int(req["steps"]), stream.cuda_stream)
        spec = s.spectra()
        launches += s.launches
        s.close()
        fin = clock() - t0
        results.append({"name": req.get("name"), "arrival_s": req["arrival_s"], "admit_s": start, "finish_s": fin,
                        "latency_s": fin - req["arrival_s"], "status": 0, "spectra": spec,
                        "cell_updates": float(np.prod(req["shape"])) * int(req["steps"])})
    wall = clock() - t0
    out = summarise(results, wall)
    out["launches"] = launches
    return results, out
