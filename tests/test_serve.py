"""The open-loop serving driver (submission at arrival times, latency from
arrival to the poll that returns the result, percentiles, refused and
failed requests) against a fake of the library's serving loop (no GPU)."""
import math

import pytest

from paper_1705_03750_gb300.serve import Request, poisson_requests, run_open_loop


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock takes a little time
        return self.t


class FakeServer:
    """Each request finishes `steps` polls after its submission; submissions
    with nx > limit are refused; request ids listed in `fail` finish with a
    non-zero status."""

    def __init__(self, clock, limit=10 ** 9, fail=()):
        self.clock, self.limit, self.fail = clock, limit, set(fail)
        self.live = {}
        self.submitted = []
        self.next = 100
        self.peak = 0

    def submit(self, cfg, f0, steps):
        if cfg[0] > self.limit:
            raise RuntimeError("vm_server_submit: memory budget exceeded (status 6)")
        rid = self.next
        self.next += 1
        self.live[rid] = [steps, cfg]
        self.submitted.append((rid, self.clock.t))
        self.peak = max(self.peak, len(self.live))
        return rid

    def poll(self):
        out = []
        for rid in list(self.live):
            self.live[rid][0] -= 1
            if self.live[rid][0] <= 0:
                del self.live[rid]
                out.append({"id": rid, "status": 5 if rid in self.fail else 0})
        return out

    def result(self, rid):
        return {"rid": rid}

    def stats(self):
        return {"peak_active": self.peak}


def test_arrivals_are_submitted_at_their_time_and_latency_counts_from_arrival():
    clock = FakeClock()
    srv = FakeServer(clock)
    reqs = [Request(0, (4, 4), steps=5, arrival=0.0), Request(1, (4, 4), steps=5, arrival=0.01)]
    rep = run_open_loop(srv, reqs, ic_fn=lambda c: None, clock=clock)
    assert rep["requests"] == 2 and rep["failed"] == 0
    t_sub = dict(srv.submitted)
    assert t_sub[101] - t_sub[100] >= 0.01 - 2e-4      # the second waited for its arrival
    r0, r1 = sorted(reqs, key=lambda r: r.rid)
    assert 0 < r0.latency < 0.01 and 0 < r1.latency < 0.01
    assert r1.latency == pytest.approx(r1.finished - 0.01)


def test_report_percentiles_and_throughput():
    clock = FakeClock()
    reqs = [Request(i, (8, 8), steps=1 + (i % 10), arrival=0.0) for i in range(100)]
    rep = run_open_loop(FakeServer(clock), reqs, ic_fn=lambda c: None, clock=clock)
    lat = sorted(r.latency for r in reqs)
    assert rep["p50_latency_s"] == lat[49] and rep["p99_latency_s"] == lat[98]
    assert rep["cell_updates_per_s"] == pytest.approx(sum(64 * r.steps for r in reqs) / rep["wall_s"])
    assert rep["peak_active"] == 100


def test_refused_and_failed_requests_are_reported_and_the_rest_complete():
    clock = FakeClock()
    srv = FakeServer(clock, limit=16, fail={102})
    reqs = [Request(i, (32 if i == 1 else 8, 8), steps=2 + i, arrival=0.0) for i in range(5)]
    rep = run_open_loop(srv, reqs, ic_fn=lambda c: None, clock=clock, keep_results=True)
    assert rep["requests"] == 5 and rep["failed"] == 2
    bad = sorted((r for r in reqs if r.error), key=lambda r: r.rid)
    assert "status 6" in bad[0].error and bad[1].error == "status 5"
    assert all(r.result for r in reqs if not r.error)


def test_poisson_requests_are_seeded():
    a = poisson_requests(20, rate=3.0, seed=7)
    b = poisson_requests(20, rate=3.0, seed=7)
    assert [(r.config, r.steps, r.arrival) for r in a] == [(r.config, r.steps, r.arrival) for r in b]
    assert all(256 <= nx <= 2048 and nx % 32 == 0 for nx, _ in (r.config for r in a))
    arr = [r.arrival for r in a]
    assert arr == sorted(arr) and not math.isnan(arr[-1])
