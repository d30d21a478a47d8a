"""Serving scheduler host logic on the CPU, with a fake executor and a simulated clock."""
import math

import pytest

from paper_1401_7494_gb300.serving import Request, Scheduler, summarize, poisson_requests


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeExecutor:
    """One device that runs submitted chunks in FIFO order at a fixed update rate."""

    def __init__(self, clock, gups=500.0, slot_bytes=lambda r: r.L ** 3 * 4 + (1 << 26), fail_on=(),
                 cache=True):
        self.clock = clock
        self.rate = gups * 1e9
        self.slot_bytes = slot_bytes
        self.fail_on = set(fail_on)
        self.device_free = 0.0
        self.held = 0            # bytes of active + cached slots
        self.peak = 0
        self.cache = cache
        self.idle = []           # cached slots: (key, bytes)
        self.opened = []

    def footprint(self, r):
        return self.slot_bytes(r)

    def cached_bytes(self):
        return sum(b for _, b in self.idle)

    def reusable(self, r):
        return any(k == (r.L, r.protocol) for k, _ in self.idle)

    def evict_idle(self, need):
        freed = 0
        while self.idle and freed < need:
            _, b = self.idle.pop(0)
            freed += b
            self.held -= b
        return freed

    def open(self, r):
        if r.rid in self.fail_on:
            raise MemoryError("injected allocation failure")
        key = (r.L, r.protocol)
        for i, (k, b) in enumerate(self.idle):
            if k == key:
                self.idle.pop(i)
                break
        else:
            self.held += self.footprint(r)
        self.peak = max(self.peak, self.held)
        self.opened.append(r.rid)
        return {"req": r, "end": 0.0, "sealed": False}

    def submit_chunk(self, h, c):
        a, b = h["req"].chunk_range(c)
        dur = h["req"].L ** 3 * (b - a) / self.rate
        start = max(self.clock(), self.device_free)
        self.device_free = start + dur
        h["end"] = self.device_free

    def seal(self, h):
        h["sealed"] = True
        h["end"] = max(h["end"], self.clock())

    def done(self, h):
        return h["sealed"] and self.clock() >= h["end"]

    def finish(self, h, keep):
        r = h["req"]
        if self.cache:
            self.idle.append(((r.L, r.protocol), self.footprint(r)))
        else:
            self.held -= self.footprint(r)
        return ("volume", r.rid) if keep else None

    def abandon(self, h):
        if not h["sealed"]:
            self.seal(h)


def run(reqs, budget=8 << 30, **kw):
    clk = SimClock()
    ex = FakeExecutor(clk, **{k: v for k, v in kw.items() if k in ("gups", "slot_bytes", "fail_on", "cache")})
    sch = Scheduler(ex, budget, max_active=kw.get("max_active", 32), clock=clk, sleep=clk.sleep,
                    keep_volumes=kw.get("keep", False))
    return sch.run(reqs), ex, sch, clk


def test_all_requests_complete_and_stats():
    reqs = poisson_requests(60, 20.0, {"p124": 124, "p248": 248}, seed=3, L_choices=(64, 128),
                            L_weights=(0.5, 0.5))
    res, ex, sch, clk = run(reqs)
    assert all(r.status == "ok" for r in res)
    s = summarize(res, reqs, clk.t)
    assert s["ok"] == 60 and s["p99_ttv_s"] >= s["p50_ttv_s"] > 0
    # every completion is after its last chunk arrived
    for q, r in zip(reqs, res):
        assert r.completed >= q.chunk_arrival(q.n_chunks - 1) - 1e-9
        assert r.admitted >= q.arrival - 1e-9


def test_memory_budget_is_never_exceeded_with_cached_slots():
    reqs = poisson_requests(80, 50.0, {"a": 64, "b": 128}, seed=4, L_choices=(128, 256, 512),
                            L_weights=(0.4, 0.4, 0.2))
    budget = 2 << 30
    res, ex, *_ = run(reqs, budget=budget)
    assert ex.peak <= budget
    assert all(r.status == "ok" for r in res)


def test_first_fit_lets_small_requests_pass_a_large_one():
    blocker = Request(0, 1024, "p", 496, arrival=0.0)        # holds ~4 GiB for a while
    big = Request(1, 1024, "p", 32, arrival=0.001)           # does not fit until the blocker is done
    small = [Request(i, 64, "p", 32, arrival=0.002 + 0.001 * i) for i in range(2, 7)]
    budget = 5 << 30
    res, ex, sch, _ = run([blocker, big] + small, budget=budget, cache=False)
    order = [rid for _, ev, rid in sch.log if ev == "admit"]
    assert order[0] == 0
    assert all(order.index(i) < order.index(1) for i in range(2, 7)), order
    assert all(r.status == "ok" for r in res)
    assert ex.peak <= budget


def test_request_larger_than_budget_is_rejected():
    res, *_ = run([Request(0, 1024, "p", 16, 0.0), Request(1, 64, "p", 16, 0.0)], budget=1 << 30)
    assert res[0].status == "rejected" and res[1].status == "ok"


def test_injected_allocation_failure_is_reported_and_isolated():
    reqs = [Request(i, 64, "p", 48, arrival=0.001 * i) for i in range(4)]
    res, ex, *_ = run(reqs, fail_on={2})
    assert [r.status for r in res] == ["ok", "ok", "error", "ok"]
    assert "allocation failed" in res[2].message


def test_stalled_producer_times_out_and_releases_memory():
    # request 0's later chunks never arrive (the producer stopped); its deadline ends it
    stalled = Request(0, 128, "p", 64, arrival=0.0, chunk_interval=math.inf, deadline=0.5)
    ok = Request(1, 128, "p", 64, arrival=0.1)
    res, ex, sch, clk = run([stalled, ok], cache=False)
    assert res[0].status == "timeout" and res[1].status == "ok"
    assert ex.held == 0                      # the stalled request's slot was released


def test_waiting_request_times_out_before_admission():
    blocker = Request(0, 512, "p", 496, arrival=0.0)
    late = Request(1, 512, "p", 496, arrival=0.01, deadline=0.05)
    budget = 512 ** 3 * 4 + (1 << 26) + (1 << 20)
    res, *_ = run([blocker, late], budget=budget, gups=100.0, cache=False)
    assert res[0].status == "ok" and res[1].status == "timeout"
    assert "not admitted" in res[1].message


def test_max_active_bounds_concurrency():
    reqs = [Request(i, 64, "p", 64, arrival=0.0) for i in range(10)]
    res, ex, sch, _ = run(reqs, max_active=3)
    live, peak = 0, 0
    for _, ev, _rid in sch.log:
        live += {"admit": 1, "done": -1}.get(ev, 0)
        peak = max(peak, live)
    assert peak <= 3 and all(r.status == "ok" for r in res)


def test_schedule_is_deterministic():
    reqs = poisson_requests(40, 30.0, {"a": 124, "b": 248}, seed=9, L_choices=(64, 128), L_weights=(0.5, 0.5))
    a = run(reqs)[2].log
    b = run(reqs)[2].log
    assert a == b


def test_overlap_stats_counts_time_with_two_requests_in_flight():
    from paper_1401_7494_gb300 import serving
    iv = [(1, 0, 0.0, 10.0), (1, 1, 10.0, 20.0), (2, 0, 5.0, 12.0), (3, 0, 30.0, 35.0), (2, 1, 12.0, 15.0)]
    st = serving.overlap_stats(iv)
    assert st["busy_ms"] == 25.0                   # [0, 20] and [30, 35]
    assert st["overlap_ms"] == 10.0                # [5, 15]: requests 1 and 2
    assert st["peak_requests_in_flight"] == 2
    assert abs(st["overlap_fraction"] - 0.4) < 1e-12
    assert serving.overlap_stats([])["busy_ms"] == 0.0
