"""Open-loop serving runs on the library's serving loop.

The scheduling itself (admission by exact workspace footprint against a
device budget, first come first served, resident state, continuous batching
of every active solve's steps into shared launches, release of finished
solves) is native code behind vm_server_* (``vlamet.NativeServer``).  This
module only drives it the way a serving front end would: requests arrive on
an open-loop schedule, each is submitted when its arrival time has come, the
server is polled, and each request's latency runs from its arrival to the
poll that hands its result over.
"""
from __future__ import annotations

import math
import statistics
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    config: object            # inputs.RunConfig
    steps: int
    arrival: float            # seconds from the start of the run
    finished: float = math.nan
    result: dict = field(default_factory=dict)
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def run_open_loop(server, requests, ic_fn, clock=time.perf_counter, keep_results: bool = False) -> dict:
    """Submit every request at its arrival time (seconds after the start),
    poll the server until all are done, and report latency percentiles
    (arrival to the poll that returned the result) and throughput."""
    pending = sorted(requests, key=lambda r: r.arrival)
    by_id = {}
    done = []
    t0 = clock()
    k = 0
    while k < len(pending) or by_id:
        now = clock() - t0
        while k < len(pending) and pending[k].arrival <= now:
            r = pending[k]
            k += 1
            try:
                by_id[server.submit(r.config, ic_fn(r.config), r.steps)] = r
            except Exception as e:  # noqa: BLE001 - a refused request is reported, the others go on
                r.error = f"{type(e).__name__}: {e}"
                r.finished = clock() - t0
                done.append(r)
        for d in server.poll():
            r = by_id.pop(d["id"])
            r.finished = clock() - t0
            if d["status"] != 0:
                r.error = f"status {d['status']}"
            elif keep_results:
                r.result = server.result(d["id"])
            done.append(r)
    wall = clock() - t0
    return report(done, wall, server.stats() if hasattr(server, "stats") else {})


def report(done, wall: float, stats: dict) -> dict:
    lat = sorted(r.latency for r in done)
    cells = sum(_sites(r.config) * r.steps for r in done if not r.error)

    def pct(p):
        if not lat:
            return math.nan
        k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]
    return {"requests": len(done), "failed": sum(1 for r in done if r.error),
            "wall_s": wall, "cell_updates_per_s": cells / wall if wall > 0 else math.nan,
            "p50_latency_s": pct(50), "p99_latency_s": pct(99),
            "mean_latency_s": statistics.fmean(lat) if lat else math.nan,
            "peak_active": stats.get("peak_active", 0), "peak_bytes": stats.get("peak_bytes", 0),
            "group_steps": stats.get("group_steps", 0)}


def _sites(cfg) -> int:
    return cfg.nx * cfg.nv if hasattr(cfg, "nx") else int(cfg[0]) * int(cfg[1])


def poisson_requests(n: int, rate: float, seed: int, sides=(256, 2048), steps=(200, 2000), make_config=None):
    """n requests with exponential inter-arrival times (rate per second),
    grid sides log-uniform in `sides` rounded to multiples of 32, and steps
    uniform in `steps`, all from `seed`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        nx = int(round(math.exp(rng.uniform(math.log(sides[0]), math.log(sides[1]))) / 32.0)) * 32
        nv = int(round(math.exp(rng.uniform(math.log(sides[0]), math.log(sides[1]))) / 32.0)) * 32
        st = int(rng.integers(steps[0], steps[1] + 1))
        cfg = make_config(i, nx, nv) if make_config else (nx, nv)
        out.append(Request(i, cfg, st, t))
    return out
