"""Host logic of the serving loop on CPU, with stand-in runs and batches (no
GPU): admission order and budget, chunked stepping to each request's budget,
a run that blows up retired as failed while the others finish, cancellation
of queued and active requests."""
import math

import pytest

from paper_2012_08758_b300 import binding as B
from paper_2012_08758_b300.serving import Request, Server


class FakeRun:
    """Grows B_rms as exp(0.1 t) with dt = 0.01; seed 666 blows up after 30 steps."""
    made = []

    def __init__(self, **p):
        self.p = p
        self.steps = 0
        self.cells = p["nx"] * p["ny"] * p["nz"]
        self.closed = False
        FakeRun.made.append(self)

    def set_seed_field(self, seed, amp):
        self.b0 = amp

    def step(self, k):
        assert not self.closed
        self.steps += k

    def time(self):
        if self.p["seed"] == 666 and self.steps >= 30:
            raise B.MhdError(B.MHD_ENONFINITE, "non-finite time step (run blew up)")
        return 0.01 * self.steps, 0.01, self.steps

    def reduce(self, kind):
        assert kind == B.MHD_BRMS
        return self.b0 * math.exp(0.1 * 0.01 * self.steps)

    def diagnostics(self):
        return {"brms": self.reduce(B.MHD_BRMS), "steps": self.steps}

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self, runs):
        self.runs = list(runs)

    def step(self, k):
        for r in self.runs:
            r.step(k)

    def close(self):
        pass


def _server(**kw):
    FakeRun.made = []
    return Server(run_factory=FakeRun, batch_factory=FakeBatch, chunk=10, **kw)


def test_runs_reach_their_budgets_and_report_growth():
    reqs = [Request(i, 0.0, 16, 50.0, 1.0, 40 + 10 * i, 100 + i) for i in range(4)]
    srv = _server()
    res = {r.id: r for r in srv.serve(reqs, realtime=False)}
    assert sorted(res) == [0, 1, 2, 3]
    for req in reqs:
        r = res[req.id]
        assert r.status == "ok" and r.diagnostics["steps"] == req.steps
        assert r.growth_rate == pytest.approx(0.1, rel=1e-9)
    assert all(run.closed for run in FakeRun.made)
    assert srv.used == 0


def test_blown_up_run_is_retired_and_the_others_finish():
    reqs = [Request(0, 0.0, 16, 50.0, 1.0, 100, 1), Request(1, 0.0, 16, 50.0, 1.0, 100, 666),
            Request(2, 0.0, 16, 50.0, 0.0, 100, 3)]
    srv = _server()
    res = {r.id: r for r in srv.serve(reqs, realtime=False)}
    assert res[1].status.startswith("failed") and "blew up" in res[1].status
    assert math.isnan(res[1].growth_rate)
    assert res[0].status == res[2].status == "ok"
    assert res[0].diagnostics["steps"] == 100 and res[2].diagnostics["steps"] == 100


def test_admission_waits_for_budget_and_slots():
    reqs = [Request(i, 0.0, 16, 50.0, 1.0, 20, 10 + i) for i in range(5)]
    srv = _server(max_active=2)
    res = srv.serve(reqs, realtime=False)
    assert [r.id for r in sorted(res, key=lambda r: r.finished)][:2] == [0, 1]
    assert max(len([1 for x in res if x.admitted <= r.admitted < x.finished]) for r in res) <= 2
    one = srv.footprint(reqs[0])
    srv2 = _server(budget_bytes=1.5 * one)  # room for one run at a time
    res2 = sorted(srv2.serve(reqs, realtime=False), key=lambda r: r.admitted)
    for a, b in zip(res2, res2[1:]):
        assert b.admitted >= a.finished


def test_cancel_drops_queued_and_retires_active():
    reqs = [Request(i, 0.0, 16, 50.0, 1.0, 200, 20 + i) for i in range(3)]
    srv = _server(max_active=1)
    srv.cancel(2)           # still queued: never admitted
    orig = srv._make_batch

    def cancel_active(runs):
        srv.cancel(0)       # active when its batch is built: retired after the chunk
        return orig(runs)

    srv._make_batch = cancel_active
    res = {r.id: r for r in srv.serve(reqs, realtime=False)}
    assert 2 not in res
    assert res[0].status == "cancelled" and res[0].diagnostics == {}
    assert res[1].status == "ok" and res[1].diagnostics["steps"] == 200
