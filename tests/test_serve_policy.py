"""The serving loop's period planner (host logic, no GPU): which admitted
requests advance in the next period."""
from paper_2005_06997_gb300.serve import plan_period


class Fake:
    def __init__(self, name, cells, remaining, last_run_s=0.0):
        self.name, self.cells, self.remaining, self.last_run_s = name, float(cells), remaining, last_run_s

    def work(self):
        return self.cells * self.remaining


def names(run):
    return sorted(a.name for a in run)


def test_small_requests_share_a_period_smallest_work_first():
    act = [Fake("big", 30e6, 8000), Fake("a", 1e6, 2000), Fake("b", 2e6, 3000), Fake("c", 4e6, 2000)]
    run = plan_period(act, now=0.1, fill_cells=16e6, max_wait_s=1.0)
    assert names(run) == ["a", "b", "c"]


def test_large_request_runs_alone_when_it_is_the_smallest_left():
    act = [Fake("big", 30e6, 100), Fake("a", 1e6, 8000)]
    run = plan_period(act, now=0.1, fill_cells=16e6, max_wait_s=1.0)
    # the big one has less remaining work (3e9 < 8e9) but does not fit with a
    assert names(run) == ["big"]


def test_fill_limit_skips_but_keeps_looking():
    act = [Fake("a", 10e6, 10), Fake("b", 10e6, 20), Fake("c", 1e6, 5000)]
    run = plan_period(act, now=0.0, fill_cells=12e6, max_wait_s=1.0)
    assert names(run) == ["a", "c"]


def test_overdue_request_joins_whatever_its_size():
    act = [Fake("big", 30e6, 8000, last_run_s=0.0), Fake("a", 1e6, 2000, last_run_s=1.9)]
    run = plan_period(act, now=2.0, fill_cells=16e6, max_wait_s=1.0)
    assert "big" in names(run)
    run = plan_period(act, now=0.5, fill_cells=16e6, max_wait_s=1.0)
    assert names(run) == ["a"]


def test_always_at_least_one():
    act = [Fake("huge", 1e9, 10)]
    assert names(plan_period(act, now=0.0, fill_cells=16e6, max_wait_s=1.0)) == ["huge"]
