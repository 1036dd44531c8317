"""Host logic of the serving loop (admission, continuous batching, chunk sizing,
divergence, latency report) against a host-only fake backend on a virtual
clock: no GPU, deterministic."""
import math

import numpy as np
import pytest

from paper_2609_24785_b300 import lee, serve, workloads


class VClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-5)


class FakeBackend:
    """Solves whose chunk takes (steps x fluid nodes) / rate seconds of
    virtual time; footprint = 100 bytes per node."""

    def __init__(self, clock, rate=1e9, diverge=(), fail_setup=()):
        self.clock, self.rate = clock, rate
        self.members = []
        self.busy_until = 0.0
        self.diverge, self.fail_setup = set(diverge), set(fail_setup)
        self.log = []                                  # (event, rid, time)
        self.chunk_members = []

    def setup(self, req):
        if req.case.name in self.fail_setup:
            raise lee.LeeError(lee.LEE_ERR_GEOMETRY, "no fluid node")
        n = req.case.nx * req.case.ny
        return object(), 100 * n, n

    def bind(self, req):
        self.log.append(("bind", req.rid, self.clock()))

    def join(self, reqs):
        for r in reqs:
            self.members.append(r)
            self.log.append(("join", r.rid, self.clock()))

    def leave(self, reqs):
        for r in reqs:
            self.members.remove(r)
            self.log.append(("leave", r.rid, self.clock()))

    def launch(self, n):
        pts = sum(r.points for r in self.members)
        self.busy_until = self.clock() + n * pts / self.rate
        self.chunk_members.append((n, [r.rid for r in self.members]))

    def done(self):
        return self.clock() >= self.busy_until

    def wait(self):
        return [lee.STATUS_DIVERGED if r.case.name in self.diverge and r.steps_done > 0 else 0
                for r in self.members]

    def result(self, req):
        return np.full((req.steps, 1), float(req.rid))

    def release(self, req):
        req.handle = None


def _case(name, n, steps):
    return workloads.Case(name, n, n, steps=steps)


def _server(clock, be, **kw):
    kw.setdefault("setup_workers", 0)
    return serve.Server(be, clock=clock, sleep=clock.sleep, rate_guess=1e9, **kw)


def test_all_requests_complete_with_exact_step_counts():
    clk = VClock()
    be = FakeBackend(clk)
    trace = [(0.001 * i, _case("r%d" % i, 64 + 32 * (i % 3), 50 + 37 * i)) for i in range(8)]
    rep = _server(clk, be, chunk_ms=5.0).run(trace)
    assert all(r.status == "ok" for r in rep.requests)
    for r in rep.requests:
        assert r.steps_done == r.steps                       # no chunk runs past a member's step count
        assert r.t_setup <= r.t_admit <= r.t_done
        assert r.latency >= r.steps * r.points / be.rate - 1e-9
    s = rep.summary()
    assert s["completed"] == 8 and s["p50_s"] <= s["p99_s"]
    assert s["mpoint_stage_per_s"] > 0
    # GPU-busy time: inside the makespan, and the busy-time rate is the higher one
    assert 0 < s["busy_s"] <= s["makespan_s"] and 0 < s["busy_share"] <= 1
    assert s["mpoint_stage_per_busy_s"] >= s["mpoint_stage_per_s"]


def test_late_arrival_joins_a_running_batch():
    """Continuous batching: a request arriving while another is on the GPU
    joins at the next chunk boundary, before the first one finishes."""
    clk = VClock()
    be = FakeBackend(clk, rate=1e7)
    trace = [(0.0, _case("long", 128, 2000)), (0.05, _case("late", 64, 100))]
    rep = _server(clk, be, chunk_ms=10.0).run(trace)
    first, late = rep.requests
    joins = {rid: t for ev, rid, t in be.log if ev == "join"}
    assert joins[late.rid] < first.t_done
    assert late.t_done < first.t_done                         # short one leaves first
    assert any(set(m) == {0, 1} for _, m in be.chunk_members)   # both in one chunk
    assert rep.peak_members == 2


def test_budget_and_slots_bound_the_resident_set():
    clk = VClock()
    be = FakeBackend(clk)
    trace = [(0.0, _case("r%d" % i, 100, 200)) for i in range(6)]  # 1e6 bytes each
    rep = _server(clk, be, budget_bytes=2_500_000).run(trace)
    assert rep.peak_bytes <= 2_500_000 and rep.peak_members == 2
    assert all(r.status == "ok" for r in rep.requests)
    clk2 = VClock()
    rep2 = _server(clk2, FakeBackend(clk2), max_slots=3).run(trace)
    assert rep2.peak_members == 3


def test_large_request_lets_small_ones_pass_a_bounded_number_of_times():
    clk = VClock()
    be = FakeBackend(clk)
    # budget 1.5e6: 'big' (1.44e6 B) fits only when nothing else is resident
    # and 'long' (resident for ~50 ms) keeps it out; the small ones fit beside 'long'
    trace = [(0.0, _case("long", 50, 20000)), (0.001, _case("big", 120, 100))] + \
            [(0.002 + 0.001 * i, _case("s%d" % i, 50, 400)) for i in range(10)]
    rep = _server(clk, be, budget_bytes=1_500_000, max_bypass=3, chunk_ms=2.0).run(trace)
    big = next(r for r in rep.requests if r.case.name == "big")
    assert big.status == "ok"
    overtook = [r for r in rep.requests if r.case.name.startswith("s") and r.t_admit < big.t_admit]
    assert len(overtook) <= 3
    assert big.bypassed == 3


def test_request_beyond_budget_and_failed_setup_are_reported():
    clk = VClock()
    be = FakeBackend(clk, fail_setup={"bad"})
    trace = [(0.0, _case("huge", 400, 10)), (0.0, _case("bad", 64, 10)), (0.0, _case("fine", 64, 10))]
    rep = _server(clk, be, budget_bytes=1_000_000).run(trace)
    st = {r.case.name: r.status for r in rep.requests}
    assert st == {"huge": "failed", "bad": "failed", "fine": "ok"}
    assert "budget" in rep.requests[0].error and "GEOMETRY" in rep.requests[1].error


def test_diverged_member_is_evicted_and_others_finish():
    clk = VClock()
    be = FakeBackend(clk, diverge={"blowup"})
    trace = [(0.0, _case("blowup", 64, 5000)), (0.0, _case("ok", 64, 300))]
    rep = _server(clk, be, chunk_ms=2.0).run(trace)
    st = {r.case.name: r for r in rep.requests}
    assert st["blowup"].status == "diverged" and st["blowup"].steps_done < 5000
    assert st["ok"].status == "ok" and st["ok"].probes is not None
    assert rep.summary()["diverged"] == 1


def test_chunk_steps_policy():
    clk = VClock()
    srv = _server(clk, FakeBackend(clk), chunk_ms=10.0)
    srv.rate = 4e9                                   # point-stages / s
    a = serve.Request(0, _case("a", 10, 1000), 0.0, steps=1000, points=100_000)
    b = serve.Request(1, _case("b", 10, 1000), 0.0, steps=1000, points=100_000)
    # 10 ms at 4e9 / (4 x 2e5 points) = 50 steps -> 48 (multiple of the graph length)
    assert srv.chunk_steps([a, b]) == 48
    b.steps_done = 990                               # b needs 10 more
    assert srv.chunk_steps([a, b]) == 10
    srv.rate = 1.0
    assert srv.chunk_steps([a]) == 1


def test_offline_trace_and_percentiles():
    clk = VClock()
    be = FakeBackend(clk)
    trace = [(10.0 * i, _case("r%d" % i, 32, 10 * (i + 1))) for i in range(5)]
    rep = _server(clk, be).run(trace, realtime=False)       # all released at once
    lat = np.sort(rep.latencies())
    assert lat.size == 5
    s = rep.summary()
    assert math.isclose(s["p50_s"], float(np.percentile(lat, 50)))
    assert s["p99_s"] <= lat[-1] + 1e-12
