"""Continuous-batching solve server over the C ABI (torch for memory and streams).

Requests (problem dicts with an ``arrival_s`` time) arrive on a clock.  The
server admits every arrived request whose state fits the HBM budget: it gets
a torch device buffer bound with ``nlf_bind_state`` and its state stays on
the device until it finishes.  Admission runs on a stream of its own while
the GPU works.

Scheduling, in two lanes on two streams that run concurrently, one DFT
period (K * B time steps) at a time per lane:
* the small lane takes the admitted requests whose grids are at most half
  of ``fill_cells``, in order of remaining work (cells x remaining steps,
  smallest first), until their grids fill ``fill_cells``; they advance
  together in one ``nlf_batch_run`` call (small grids leave most of the GPU
  idle on their own);
* the large lane advances one larger request at a time through ``nlf_run``
  (the single-grid kernels), the one with the least remaining work.
A lane plans its next period as soon as its last one has finished, so small
requests are never held to a large grid's step rate and large requests keep
advancing while small ones come and go.  Within a lane a request that has
not advanced for ``max_wait_s`` goes first.  Requests that arrive while
others run join at their lane's next period; finished requests are retired
there, their spectra copied out and their memory returned.  ``cancel`` drops
a waiting request or retires an admitted one at its next period boundary.

``serve_fifo`` is the plain form for comparison: one request at a time, in
arrival order, one grid per launch sequence.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import nlfdtd

CANCELLED = -100          # status of a cancelled request


class _Active:
    __slots__ = ("req", "solver", "buf", "remaining", "admit_s", "last_run_s", "cells", "cancelled")

    def __init__(self, req, solver, buf, admit_s):
        self.req = req
        self.solver = solver
        self.buf = buf
        self.remaining = int(req["steps"])
        self.admit_s = admit_s
        self.last_run_s = admit_s
        self.cells = float(np.prod(req["shape"]))
        self.cancelled = False

    def work(self):
        return self.cells * self.remaining


def _percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def summarise(results, wall_s):
    done = [r for r in results if r["status"] == 0]
    lat = [r["latency_s"] for r in done]
    work = sum(r["cell_updates"] for r in done)
    return {"solves": len(done), "wall_s": wall_s, "solves_per_s": len(done) / wall_s if wall_s > 0 else None,
            "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
            "gcell_updates_per_s": work / wall_s / 1e9 if wall_s > 0 else None}


def plan_period(active, now, fill_cells, max_wait_s):
    """The requests that advance in the next period: those waiting longer
    than max_wait_s first, then the others by remaining work, smallest
    first, while the grids' cells stay within fill_cells (at least one
    request always runs).  A request larger than fill_cells runs alone
    unless an overdue request joins it.  Host logic only."""
    overdue = [a for a in active if now - a.last_run_s > max_wait_s]
    rest = sorted((a for a in active if now - a.last_run_s <= max_wait_s), key=lambda a: a.work())
    run = list(overdue)
    cells = sum(a.cells for a in run)
    for a in rest:
        if run and cells + a.cells > fill_cells:
            continue
        run.append(a)
        cells += a.cells
    return run


class Server:
    def __init__(self, hbm_budget_bytes: int, max_active: int = 256, stream=None, fill_cells: float = 4e6,
                 max_wait_s: float = 1.5, period_b: int = 16):
        import torch
        nlfdtd.require_gpu()
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream2 = torch.cuda.Stream()
        self.init_stream = torch.cuda.Stream()
        self.fill_cells = float(fill_cells)
        self.max_wait_s = float(max_wait_s)
        self.period_b = int(period_b)
        self.used = 0
        self.launches = 0
        self._cancel = set()

    def cancel(self, name):
        """Cancel the request called `name`: dropped if still waiting, retired
        at the next period boundary if admitted (status CANCELLED)."""
        self._cancel.add(name)

    def _admit(self, req, now):
        s = nlfdtd.Solver(req, block_b=self.period_b)
        nb = s.state_bytes()
        buf = self.torch.empty(nb + 256, dtype=self.torch.uint8, device="cuda")
        ptr = (buf.data_ptr() + 255) // 256 * 256
        s.bind_state(ptr, nb)
        s.reset(self.init_stream.cuda_stream)
        self.used += nb
        return _Active(req, s, buf, now)

    def _admit_waiting(self, waiting, active, sizes, now, results):
        """Admit waiting requests in arrival order by HBM budget and slots; a
        request larger than the whole budget is refused (NLF_E_OOM)."""
        while waiting and len(active) < self.max_active:
            req = waiting[0]
            if req.get("name") in self._cancel:
                waiting.popleft()
                results.append(_result(req, None, now, CANCELLED))
                continue
            key = id(req)
            if key not in sizes:
                probe = nlfdtd.Solver(req, block_b=self.period_b)
                sizes[key] = probe.state_bytes()
                probe.close()
            if sizes[key] > self.budget:
                waiting.popleft()
                results.append(_result(req, None, now, -4))
                continue
            if self.used + sizes[key] > self.budget:
                break
            waiting.popleft()
            active.append(self._admit(req, now))

    def run(self, requests, clock=time.perf_counter):
        """Serve `requests` (sorted by arrival_s); returns (results, summary)."""
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival_s"]))
        waiting = collections.deque()
        active = []
        results = []
        t0 = clock()
        sizes = {}
        torch = self.torch
        lanes = [_Lane(self.stream, small=True), _Lane(self.stream2, small=False)]
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0]["arrival_s"] <= now:
                waiting.append(pending.popleft())
            if waiting:
                self._admit_waiting(waiting, active, sizes, now, results)
            # retire the work of lanes whose period has finished
            for lane in lanes:
                if lane.ev is not None and lane.ev.query():
                    active = self._finish(lane, active, clock() - t0, results)
            # cancelled requests that are not running leave now
            busy = {id(a) for lane in lanes if lane.ev is not None for a in lane.run}
            gone = {id(a) for a in active if id(a) not in busy and a.req.get("name") in self._cancel}
            if gone:
                now = clock() - t0
                for a in active:
                    if id(a) in gone:
                        results.append(_result(a.req, a.admit_s, now, CANCELLED))
                active = self._retire(active, gone)
            # plan and launch the idle lanes
            launched = False
            for lane in lanes:
                if lane.ev is not None:
                    continue
                free = [a for a in active if id(a) not in busy and (a.cells <= self.fill_cells / 2) == lane.small]
                if not free:
                    continue
                if lane.small:
                    run = plan_period(free, now, self.fill_cells, self.max_wait_s)
                else:
                    run = plan_period(free, now, 0.0, self.max_wait_s)[:1]
                U = _period(run[0], self.period_b)
                lane.run = run
                lane.steps = [min(U, a.remaining) for a in run]
                lane.before = sum(a.solver.launches for a in run)
                if len(run) == 1:
                    run[0].solver.run(lane.steps[0], lane.stream.cuda_stream)
                    lane.status = [0]
                else:
                    lane.status = nlfdtd.batch_run([a.solver for a in run], lane.steps, lane.stream.cuda_stream)
                lane.ev = torch.cuda.Event()
                lane.ev.record(lane.stream)
                busy.update(id(a) for a in run)
                launched = True
            if not launched:
                if all(lane.ev is None for lane in lanes):
                    if pending and not waiting:
                        time.sleep(max(0.0, min(0.05, pending[0]["arrival_s"] - (clock() - t0))))
                else:
                    time.sleep(0.0002)
        wall = clock() - t0
        return results, summarise(results, wall)

    def _finish(self, lane, active, now, results):
        """Account a lane's finished period; retire finished and cancelled
        requests (also cancelled ones that did not run).  Returns the active
        list without them."""
        self.launches += sum(a.solver.launches for a in lane.run) - lane.before
        done = set()
        for a, n, st in zip(lane.run, lane.steps, lane.status):
            a.remaining -= n
            a.last_run_s = now
            cancelled = a.req.get("name") in self._cancel
            if st != 0 or a.remaining <= 0 or cancelled:
                code = CANCELLED if cancelled and st == 0 and a.remaining > 0 else int(st)
                res = _result(a.req, a.admit_s, now, code)
                if code == 0:
                    res["spectra"] = a.solver.spectra()
                results.append(res)
                done.add(id(a))
        lane.ev = None
        lane.run = []
        return self._retire(active, done)

    def _retire(self, active, done):
        for a in active:
            if id(a) in done:
                self.used -= a.solver.state_bytes()
                a.solver.close()
                a.buf = None
        return [a for a in active if id(a) not in done]


class _Lane:
    """One stream of the server and the period it has in flight."""

    def __init__(self, stream, small):
        self.stream = stream
        self.small = small
        self.ev = None
        self.run = []
        self.steps = []
        self.status = []
        self.before = 0


def _result(req, admit_s, now, status):
    return {"name": req.get("name"), "arrival_s": req["arrival_s"], "admit_s": admit_s, "finish_s": now,
            "latency_s": now - req["arrival_s"], "status": int(status),
            "cell_updates": float(np.prod(req["shape"])) * int(req["steps"])}


# Samples buffered per DFT flush for served requests (the default of
# Server.period_b): a period is one DFT period (K * B steps), so this sets
# how often finished requests leave and new ones join.
SERVE_B = 16


def _period(a, b=SERVE_B):
    """Time steps of one DFT period of an active request (the scheduling unit)."""
    mon = a.req.get("monitors")
    K = mon.get("K", 16) if mon else 1
    kb = K * b
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
        r = _result(req, start, fin, 0)
        r["spectra"] = spec
        results.append(r)
    wall = clock() - t0
    out = summarise(results, wall)
    out["launches"] = launches
    return results, out
