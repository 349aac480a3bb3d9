"""Serving many solves with continuous batching.

Requests (one solve each: a grid, an initial condition, a number of steps)
arrive over time.  The server admits a waiting request as soon as a slot and
enough device memory are free (admission by the solve's exact workspace
footprint against a budget), keeps every admitted solve's state resident on
the device, and advances all active solves together: each owns a CUDA
stream, and each scheduling tick queues a few steps of every active solve, so
the work of different requests overlaps on the GPU.  A solve gets new steps
only while fewer than two of its earlier chunks are still queued, so that one
host thread keeps every stream fed instead of blocking on a full launch
queue.  A solve that has queued
all its steps records an event; when the event has completed its result (the
density and force of the last step) is read back, its latency recorded and
its memory and slot released for the next request.

The scheduling logic is separate from the device backend, so it can be
exercised with a fake backend on a machine without a GPU.
"""
from __future__ import annotations

import collections
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
    admitted: float = math.nan
    finished: float = math.nan
    result: dict = field(default_factory=dict)
    error: str = ""           # set if the solve failed (its result is then empty)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class GpuBackend:
    """Solves on the current CUDA device through the C ABI: one Solver and one
    stream per request."""

    def __init__(self, precision=None, device=None):
        import torch
        from . import vlamet as V
        self.torch, self.V = torch, V
        self.precision = V.VM_FP32_MIXED if precision is None else precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())

    def footprint(self, rc) -> int:
        return self.V.workspace_bytes(self.V.Config.from_run(rc, self.precision)) + 8 * rc.nx * rc.nv

    # steps queued ahead per solve: one host thread feeds every stream, and a
    # launch into a full queue would block it while the other streams drain
    MAX_IN_FLIGHT = 2

    def start(self, req: Request, f0: np.ndarray):
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        solver = self.V.Solver(self.V.Config.from_run(req.config, self.precision), stream=stream, device=self.device)
        with torch.cuda.stream(stream):
            f_dev = torch.from_numpy(f0).to(self.device, non_blocking=False)
        solver.set_f(f_dev)
        return {"solver": solver, "stream": stream, "left": req.steps, "event": None, "f": f_dev,
                "inflight": collections.deque()}

    def ready(self, handle) -> bool:
        q = handle["inflight"]
        while q and q[0].query():
            q.popleft()
        return len(q) < self.MAX_IN_FLIGHT

    def advance(self, handle, n: int) -> None:
        handle["solver"].step(n)
        handle["left"] -= n
        ev = self.torch.cuda.Event()
        ev.record(handle["stream"])
        handle["inflight"].append(ev)
        if handle["left"] == 0:
            handle["event"] = ev

    def done(self, handle) -> bool:
        return handle["event"] is not None and handle["event"].query()

    def result(self, handle) -> dict:
        return handle["solver"].density_force()

    def release(self, handle) -> None:
        handle["solver"].close()
        handle.clear()


class Server:
    """Continuous batching of solves under a device-memory budget."""

    def __init__(self, backend, budget_bytes: int, max_active: int = 64, steps_per_tick: int = 1,
                 ic_fn=None, clock=time.perf_counter):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.steps_per_tick = int(steps_per_tick)
        self.ic_fn = ic_fn
        self.clock = clock
        self.waiting: collections.deque = collections.deque()
        self.active: list = []
        self.done: list = []
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0
        self.t0 = None

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request) -> None:
        need = self.backend.footprint(req.config)
        if need > self.budget:
            raise ValueError(f"request {req.rid} needs {need} bytes, more than the whole budget {self.budget}")
        self.waiting.append(req)

    def _admit(self) -> None:
        # first come, first served: a request that does not fit blocks the
        # ones behind it (no overtaking, so latencies stay fair)
        while self.waiting and len(self.active) < self.max_active:
            req = self.waiting[0]
            if req.arrival > self.now():
                break
            need = self.backend.footprint(req.config)
            if self.used + need > self.budget:
                break
            self.waiting.popleft()
            req.admitted = self.now()
            try:
                f0 = self.ic_fn(req.config) if self.ic_fn else None
                handle = self.backend.start(req, f0)
            except Exception as e:  # noqa: BLE001
                req.error = f"{type(e).__name__}: {e}"
                req.finished = self.now()
                self.done.append(req)
                continue
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.active.append((req, handle, need))
        self.peak_active = max(self.peak_active, len(self.active))

    def _tick(self) -> None:
        for req, handle, _ in self.active:
            left = handle["left"]
            ready = getattr(self.backend, "ready", None)
            if left > 0 and not req.error and (ready is None or ready(handle)):
                try:
                    self.backend.advance(handle, min(self.steps_per_tick, left))
                except Exception as e:  # noqa: BLE001
                    req.error = f"{type(e).__name__}: {e}"
        still = []
        for req, handle, need in self.active:
            if req.error or (handle["left"] == 0 and self.backend.done(handle)):
                # a failed solve is reported on its request; the others go on
                if not req.error:
                    try:
                        req.result = self.backend.result(handle)
                    except Exception as e:  # noqa: BLE001
                        req.error = f"{type(e).__name__}: {e}"
                req.finished = self.now()
                self.backend.release(handle)
                self.used -= need
                self.done.append(req)
            else:
                still.append((req, handle, need))
        self.active = still

    def run(self, requests, idle_sleep: float = 0.0) -> dict:
        """Serve `requests` (arrival times relative to now) until all are done."""
        self.t0 = self.clock()
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        while self.waiting or self.active:
            self._admit()
            if self.active:
                self._tick()
            elif self.waiting and idle_sleep:
                time.sleep(idle_sleep)
        wall = self.now()
        return self.report(wall)

    def report(self, wall: float) -> dict:
        lat = sorted(r.latency for r in self.done)
        cells = sum(_sites(r.config) * r.steps for r in self.done)

        def pct(p):
            if not lat:
                return math.nan
            k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
            return lat[k]
        return {"requests": len(self.done), "failed": sum(1 for r in self.done if r.error),
                "wall_s": wall, "cell_updates_per_s": cells / wall if wall > 0 else math.nan,
                "p50_latency_s": pct(50), "p99_latency_s": pct(99),
                "mean_latency_s": statistics.fmean(lat) if lat else math.nan,
                "peak_active": self.peak_active, "peak_bytes": self.peak_used}


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
