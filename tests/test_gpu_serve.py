"""Serving: continuous batching with HBM-budget admission (serve.Server)
against the same requests solved alone, and the FIFO one-at-a-time form."""
import copy

import numpy as np
import pytest

from paper_2005_06997_gb300 import nlfdtd, serve
from paper_2005_06997_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_requests(n, max_side=72, nf=24, spread_s=0.2):
    reqs = []
    for r in W.serving_requests(nf=nf):
        if r["shape"][0] <= max_side:
            q = copy.deepcopy(r)
            q["steps"] = min(q["steps"], 2600)
            reqs.append(q)
        if len(reqs) == n:
            break
    # arrivals spread over spread_s so that later requests join a running batch
    for q, t in zip(reqs, np.linspace(0.0, spread_s, len(reqs))):
        q["arrival_s"] = float(t)
    return reqs


def alone_spectra(req):
    s = nlfdtd.Solver(req)
    s.run(req["steps"])
    sp = s.spectra()
    s.close()
    return sp


def assert_close(sp, ref, tol=1e-4):
    for key in ("ext", "abs", "sca"):
        scale = np.max(np.abs(ref[key]))
        assert np.max(np.abs(sp[key] - ref[key])) <= tol * scale, key


def test_served_results_equal_alone_results():
    reqs = small_requests(6)
    srv = serve.Server(hbm_budget_bytes=64 << 30)
    results, summary = srv.run(reqs)
    assert summary["solves"] == len(reqs)
    by_name = {r["name"]: r for r in results}
    for q in reqs:
        r = by_name[q["name"]]
        assert r["status"] == 0
        assert r["latency_s"] >= 0 and r["finish_s"] >= q["arrival_s"]
        assert_close(r["spectra"], alone_spectra(q))
    assert srv.launches > 0


def test_admission_respects_hbm_budget():
    reqs = small_requests(5)
    sizes = []
    for q in reqs:
        s = nlfdtd.Solver(q)
        sizes.append(s.state_bytes())
        s.close()
    budget = 2 * max(sizes) + 1            # at most two requests resident at once
    srv = serve.Server(hbm_budget_bytes=budget)
    peak = {"used": 0}
    orig = srv._admit

    def admit(req, now):
        a = orig(req, now)
        peak["used"] = max(peak["used"], srv.used)
        return a

    srv._admit = admit
    results, summary = srv.run(reqs)
    assert summary["solves"] == len(reqs)
    assert peak["used"] <= budget
    assert srv.used == 0


def test_fifo_matches_batched():
    reqs = small_requests(3)
    res_b, _ = serve.Server(hbm_budget_bytes=64 << 30).run(reqs)
    res_f, summ_f = serve.serve_fifo(reqs)
    fb = {r["name"]: r for r in res_b}
    for r in res_f:
        assert_close(r["spectra"], fb[r["name"]]["spectra"])
    assert summ_f["solves"] == 3


@pytest.mark.parametrize("when", ["waiting", "running"])
def test_cancelled_request_leaves_the_others_unchanged(when):
    """A request cancelled before it is admitted is dropped; one cancelled
    while it runs (here: when the next request is admitted) is retired at
    the next period boundary.  The others finish as they would alone."""
    reqs = small_requests(5, spread_s=0.05)
    victim = reqs[2]["name"]
    srv = serve.Server(hbm_budget_bytes=64 << 30)
    if when == "waiting":
        srv.cancel(victim)
    else:
        orig = srv._admit

        def admit(req, now):
            a = orig(req, now)
            if req["name"] == reqs[3]["name"]:
                srv.cancel(victim)
            return a

        srv._admit = admit
    results, summary = srv.run(reqs)
    by_name = {r["name"]: r for r in results}
    assert by_name[victim]["status"] == serve.CANCELLED
    assert "spectra" not in by_name[victim]
    assert summary["solves"] == len(reqs) - 1
    for q in reqs:
        if q["name"] != victim:
            assert_close(by_name[q["name"]]["spectra"], alone_spectra(q))
    assert srv.used == 0


def test_request_larger_than_the_budget_is_refused():
    reqs = small_requests(3)
    sizes = []
    for q in reqs:
        s = nlfdtd.Solver(q, block_b=serve.SERVE_B)      # as the server sizes them
        sizes.append(s.state_bytes())
        s.close()
    big = int(np.argmax(sizes))
    srv = serve.Server(hbm_budget_bytes=max(sizes) - 1)
    results, summary = srv.run(reqs)
    by_name = {r["name"]: r for r in results}
    assert by_name[reqs[big]["name"]]["status"] == -4        # NLF_E_OOM
    assert summary["solves"] == len(reqs) - 1
    assert srv.used == 0


def test_two_lanes_side_by_side_equal_alone_results(monkeypatch):
    """With fill_cells set so that about half of the requests count as large,
    the large lane (one grid at a time through nlf_run) and the small lane
    (batches through nlf_batch_run) run side by side on two non-blocking
    streams while requests come and go, each lane making new batched plans
    and graphs as its member set changes: every served result equals the
    request solved alone."""
    reqs = small_requests(10, spread_s=0.02)
    fill = 4.4e5
    n_large = sum(1 for q in reqs if np.prod(q["shape"]) > fill / 2)
    assert 3 <= n_large <= 7
    sizes = []
    orig = nlfdtd.batch_run

    def batch_run(solvers, steps, stream=None):
        sizes.append(len(solvers))
        return orig(solvers, steps, stream)

    monkeypatch.setattr(nlfdtd, "batch_run", batch_run)
    srv = serve.Server(hbm_budget_bytes=64 << 30, fill_cells=fill)
    results, summary = srv.run(reqs)
    assert summary["solves"] == len(reqs)
    assert max(sizes) >= 2                       # the small lane batched
    by_name = {r["name"]: r for r in results}
    for q in reqs:
        r = by_name[q["name"]]
        assert r["status"] == 0
        assert_close(r["spectra"], alone_spectra(q))
    assert srv.used == 0
