"""Scheduling of the serving layer with a fake device backend (no GPU)."""
import math

import pytest

from paper_1705_03750_gb300.serve import Request, Server, poisson_requests


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Each request's footprint is nx*nv bytes; a step of a request takes one
    tick; the clock advances 1 per tick."""

    def __init__(self, clock):
        self.clock = clock
        self.log = []

    def footprint(self, cfg):
        return cfg[0] * cfg[1]

    def start(self, req, f0):
        self.log.append(("start", req.rid, self.clock.t))
        return {"left": req.steps, "rid": req.rid}

    def advance(self, h, n):
        h["left"] -= n
        self.clock.t += 0.001

    def done(self, h):
        return h["left"] == 0

    def result(self, h):
        return {"rid": h["rid"]}

    def release(self, h):
        self.log.append(("end", h["rid"], self.clock.t))


def test_budget_and_slots_bound_the_active_set():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, budget_bytes=100, max_active=3, clock=clock)
    reqs = [Request(i, (5, 10), steps=3 + i, arrival=0.0) for i in range(8)]   # 50 B each
    rep = srv.run(reqs)
    assert rep["requests"] == 8
    assert srv.peak_used <= 100 and srv.peak_active <= 2       # the budget binds before the slots
    assert all(r.result["rid"] == r.rid for r in srv.done)
    # first come, first served
    starts = [rid for kind, rid, _ in be.log if kind == "start"]
    assert starts == sorted(starts)


def test_arrivals_wait_for_their_time_and_latency_counts_from_arrival():
    clock = FakeClock()
    be = FakeBackend(clock)

    class TickingBackend(FakeBackend):
        pass

    srv = Server(be, budget_bytes=10 ** 6, max_active=8, clock=clock)
    reqs = [Request(0, (4, 4), steps=5, arrival=0.0), Request(1, (4, 4), steps=5, arrival=0.003)]

    # advance the clock while idle so that the second arrival comes due
    orig = srv._admit

    def admit():
        if not srv.active and srv.waiting:
            clock.t += 0.001
        orig()
    srv._admit = admit
    srv.run(reqs)
    r0, r1 = sorted(srv.done, key=lambda r: r.rid)
    assert r1.admitted >= 0.003 - 1e-12
    assert r0.latency > 0 and r1.latency > 0
    assert r1.latency == pytest.approx(r1.finished - 0.003)


def test_request_larger_than_the_budget_is_refused():
    clock = FakeClock()
    srv = Server(FakeBackend(clock), budget_bytes=10, clock=clock)
    with pytest.raises(ValueError):
        srv.submit(Request(0, (10, 10), steps=1, arrival=0.0))


def test_report_percentiles():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, budget_bytes=10 ** 9, max_active=100, clock=clock)
    reqs = [Request(i, (8, 8), steps=1 + (i % 10), arrival=0.0) for i in range(100)]
    rep = srv.run(reqs)
    lat = sorted(r.latency for r in srv.done)
    assert rep["p50_latency_s"] == lat[49] and rep["p99_latency_s"] == lat[98]
    assert rep["cell_updates_per_s"] > 0


def test_poisson_requests_are_seeded():
    a = poisson_requests(20, rate=3.0, seed=7)
    b = poisson_requests(20, rate=3.0, seed=7)
    assert [(r.config, r.steps, r.arrival) for r in a] == [(r.config, r.steps, r.arrival) for r in b]
    assert all(256 <= nx <= 2048 and nx % 32 == 0 for nx, _ in (r.config for r in a))
    arr = [r.arrival for r in a]
    assert arr == sorted(arr) and not math.isnan(arr[-1])


def test_a_failed_solve_is_reported_and_the_rest_complete():
    clock = FakeClock()

    class Failing(FakeBackend):
        def result(self, h):
            if h["rid"] == 2:
                raise RuntimeError("device status 5")
            return super().result(h)

    srv = Server(Failing(clock), budget_bytes=10 ** 6, max_active=4, clock=clock)
    rep = srv.run([Request(i, (4, 4), steps=2 + i, arrival=0.0) for i in range(5)])
    assert rep["requests"] == 5 and rep["failed"] == 1
    bad = [r for r in srv.done if r.error]
    assert [r.rid for r in bad] == [2] and "status 5" in bad[0].error and bad[0].result == {}
    assert srv.used == 0


def test_a_solve_that_fails_while_stepping_is_retired():
    clock = FakeClock()

    class Failing(FakeBackend):
        def advance(self, h, n):
            if h["rid"] == 1 and h["left"] < 4:
                raise RuntimeError("vm_step: CUDA runtime error")
            super().advance(h, n)

    srv = Server(Failing(clock), budget_bytes=10 ** 6, max_active=2, clock=clock)
    rep = srv.run([Request(i, (4, 4), steps=6, arrival=0.0) for i in range(4)])
    assert rep["requests"] == 4 and rep["failed"] == 1
    assert [r.rid for r in srv.done if r.error] == [1] and srv.used == 0


def test_a_request_that_cannot_start_is_retired():
    clock = FakeClock()

    class Refusing(FakeBackend):
        def start(self, req, f0):
            if req.rid == 0:
                raise ValueError("expected an array of shape (4, 4)")
            return super().start(req, f0)

    srv = Server(Refusing(clock), budget_bytes=10 ** 6, max_active=2, clock=clock)
    rep = srv.run([Request(i, (4, 4), steps=3, arrival=0.0) for i in range(3)])
    assert rep["requests"] == 3 and rep["failed"] == 1 and srv.used == 0


def test_solves_that_are_not_ready_are_skipped_in_a_tick():
    clock = FakeClock()

    class Busy(FakeBackend):
        def __init__(self, clock):
            super().__init__(clock)
            self.asked = 0

        def ready(self, h):
            self.asked += 1
            return self.asked % 2 == 0     # every other query says "still busy"

    be = Busy(clock)
    srv = Server(be, budget_bytes=10 ** 6, max_active=3, clock=clock)
    rep = srv.run([Request(i, (4, 4), steps=4, arrival=0.0) for i in range(3)])
    assert rep["requests"] == 3 and rep["failed"] == 0 and be.asked > 12
