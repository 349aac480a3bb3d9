#!/usr/bin/env python
"""Benchmark of the metric semi-Lagrangian Vlasov-Poisson step on GB300.

Metric: cell-updates/s (one grid site reconstructed in one time step; the
remap every n_s steps is inside the timed steps) on the 4096 x 4096 halo
workload (16 warm Gaussian halos, elements every 8 sites, dt = 0.002,
remap every 25 steps), FP32-mixed path as the headline and the FP64 path
beside it.  Synthetic seeded input; working set > L2, so no flush between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU (torchrun): every rank advances its own independent solve (the
method has no data-parallel exchange for independent problems: replicas,
weak scaling); the timed region is bracketed by a barrier and a device
synchronisation on every rank and the max over ranks is reported.

--impl reference times the FP64 CPU oracle (the plain restatement of the
paper used by the tests) on this machine's host cores on the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1705_03750_gb300 import inputs as I  # noqa: E402

METRIC = "cell-updates/s at 4096^2 (FP32 vs FP64 path)"
WORKLOAD = I.HALOS_4096


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock and throttle samples every 20 ms, read by a thread
    that stamps each line with the host clock: started before the warm-up
    (its start-up takes longer than a short timed region), the summary keeps
    the samples that arrived while the timed region ran (mark_begin to
    mark_end, plus one interval of reporting slack)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_id: str, path: str | None = None):
        self.gpu_id, self.path, self.proc = gpu_id, path, None
        self.lines, self.t_begin, self.t_end, self.thread = [], None, None, None

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
                 str(self.INTERVAL_MS), "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except Exception:
            self.proc = None
            return self

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))
        self.thread = threading.Thread(target=read, daemon=True)
        self.thread.start()
        return self

    def mark_begin(self):
        self.t_begin = time.perf_counter()

    def mark_end(self):
        self.t_end = time.perf_counter()

    def stop(self):
        if self.proc is not None:
            time.sleep(2 * self.INTERVAL_MS / 1e3)  # the samples of the region's last interval
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=5)
        if self.path:
            with open(self.path, "a") as fh:
                fh.write("".join(f"{t:.4f},{ln}" for t, ln in self.lines))

    def __enter__(self):
        self.start()
        self.mark_begin()
        return self

    def __exit__(self, *exc):
        self.mark_end()
        self.stop()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t_begin if self.t_begin is not None else float("-inf")
        hi = (self.t_end if self.t_end is not None else float("inf")) + self.INTERVAL_MS / 1e3
        inside = [ln for t, ln in self.lines if lo <= t <= hi]
        if not inside:  # a region shorter than the sampler's first interval: the next sample
            after = [ln for t, ln in self.lines if t >= lo]
            inside = after[:1]
        for line in inside:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per kernel launch (see the design notes)
# ---------------------------------------------------------------------------

def algorithmic(kernel: str, rc, fp32: bool, ne: int):
    """(bytes, unit count, per-unit description) of one launch: the bytes the
    method must move at minimum, independent of how the kernel moves them."""
    n = rc.nx * rc.nv
    sr = 4 if fp32 else 8
    tay = 16 * 8
    if kernel == "reconstruct":
        # map 4 + f_ini 1x + f 1x per site, Taylor records once per element
        return n * (4 + 2 * sr) + ne * tay, n, f"{4 + 2 * sr} B/site + 128 B/element"
    if kernel == "remap_resample":
        return n * (4 + 2 * sr) + ne * tay, n, f"{4 + 2 * sr} B/site + 128 B/element"
    if kernel in ("claim_pair", "claim_small", "claim_large"):
        # the influence map written once (4 B/site), each element's record read once
        return n * 4 + ne * tay, n, "4 B/site + 128 B/element"
    if kernel in ("spline_rows", "spline_cols"):
        return n * 4 * sr, n, f"{4 * sr} B/site (2 sweeps, read+write)"
    if kernel in ("drift_taylor", "kick_drift"):
        return ne * (24 * 8 + (tay if kernel == "drift_taylor" else 0)), ne, "element state r+w"
    return None


# FP64 floating-point operations per site of the FP64 path's reconstruction
# on its certified branch (a fused multiply-add counts 2): site position 2,
# P - P_m 2, the second-order offset Q - Q_m 36, the anchored index
# coordinates 4, the offsets from the nodes 2, the six-point value 29.
FP64_FLOPS_PER_SITE = 75


def fp64_roofline(sites: int, avg_s: float) -> dict:
    """The FP64 reconstruction against the FP64 arithmetic peak measured on
    this device in the same run (vm_measure_fp64_peak: FMA chains, 2 FLOP per
    FMA)."""
    from paper_1705_03750_gb300 import vlamet as V
    peak = V.measure_fp64_peak(20000)
    ach = FP64_FLOPS_PER_SITE * sites / avg_s
    return {"kernel": "reconstruct", "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
            "unit": "TFLOP/s (FP64)", "frac": ach / peak, "per_unit": f"{FP64_FLOPS_PER_SITE} FP64 FLOP/site",
            "units": sites, "avg_ms": avg_s * 1e3, "peak_kind": "measured in this run (FMA chains)"}


def step_bytes_per_update(rc, fp32: bool) -> float:
    """Algorithmic bytes of one cell update of the whole step: f_ini read and
    f written once, the element state read and written once per element
    (304 B over s^2 sites), the map written and read once (8 B), and the
    remap's 24 B per site amortised over n_s steps."""
    sr = 4 if fp32 else 8
    return 2 * sr + 304.0 / (rc.s * rc.s) + 8 + 24.0 / rc.n_s


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernels captured with ncu on the 4096^2 workload (the captures summarised
# under profiles/), with the SHA-256 prefix of the kernel's source file at the
# time of the capture: a source changed since makes the figure void (null).
NCU_TRAFFIC = {
    # kernel: (bytes per launch, source file, sha256 prefix)
    "claim_pair": (137_759_488, "map.cu", "7ef7750fd3fe8b25"),
    "reconstruct": (219_803_904, "recon.cu", "69a045f1457ded49"),
}

# Warp instructions per launch (smsp__inst_executed.sum) from the same
# captures, for the kernels bound by instruction issue rather than by DRAM:
# their issue roofline is these instructions over the launch time against
# one warp instruction per scheduler per clock (4 schedulers x 152 SMs).
NCU_INSTR = {
    "claim_pair": (373_507_280, "map.cu", "7ef7750fd3fe8b25"),
    "reconstruct": (126_116_341, "recon.cu", "69a045f1457ded49"),
}
SCHEDULERS = 4 * 152

# The same figures for the 4D phase-space path's dominant kernel, captured on
# its 64^4 workload (profiles/percolate4d_halos4d64_fp64.md).  The key hashes
# the source up to the start of its reconstruction section: the percolation
# kernels and everything they use come before it in the translation unit, so
# changes further down cannot change their code.
PHASE4D_PREFIX_END = "// Sec. 2.2.1: 15-point quadratic interpolation; transport reconstruction"
NCU4_TRAFFIC = {"percolate": (236_288_768, "phase4d.cu", "908be1a679b46900")}
NCU4_INSTR = {"percolate": (4_068_047_765, "phase4d.cu", "908be1a679b46900")}


def issue_roofline(kernel: str, avg_s: float, sm_mhz):
    """Issue roofline of a kernel with a captured instruction count, or None."""
    n = _keyed(NCU_INSTR, kernel)
    if n is None or not sm_mhz:
        return None
    peak = SCHEDULERS * sm_mhz * 1e6
    ach = n / avg_s
    return {"warp_instructions": n, "achieved": ach, "peak": peak, "unit": "warp-instr/s",
            "frac": ach / peak, "clock_mhz": sm_mhz}


def ncu_traffic(kernel: str):
    return _keyed(NCU_TRAFFIC, kernel)


def _keyed(table, kernel: str, prefix_end: str | None = None):
    """The table's figure for `kernel` if its source still hashes to the
    captured key (the whole file, or its text before the line `prefix_end`,
    the start of the section's rule line above it), else None."""
    ent = table.get(kernel)
    if not ent:
        return None
    nbytes, src, sha = ent
    import hashlib
    path = os.path.join(ROOT, "paper_1705_03750_gb300", "csrc", src)
    try:
        with open(path, "rb") as fh:
            text = fh.read()
    except OSError:
        return None
    if prefix_end is not None:
        i = text.find(prefix_end.encode())
        if i < 0:
            return None
        text = text[:text.rindex(b"\n// ----", 0, i)]
    h = hashlib.sha256(text).hexdigest()
    return nbytes if h.startswith(sha) else None


# ---------------------------------------------------------------------------
# replicas over ranks (one independent solve per GPU)
# ---------------------------------------------------------------------------

def rank_workload(rank: int):
    """Rank r advances its own solve of the workload, seeded seed + r."""
    return WORKLOAD.with_(seed=WORKLOAD.seed + rank)


def max_over_ranks(x: float, dist, device) -> float:
    """Slowest rank's value (all ranks get it); identity without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, sites: int, steps: int, ms_max: float) -> float:
    """Whole-job cell updates per second: every rank's sites over the slowest
    rank's time."""
    return world * sites * steps / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def e2e_run(V, rc, prec, f0, args, dev, barrier, max_ranks, world):
    """End-to-end rate through the C ABI with host buffers.  The upload of
    f0 (vm_set_f from pinned host memory) and the K timed steps, each
    followed by vm_density_force into pinned host buffers, are timed on the
    host clock; the W warm-up steps between them are not, so the timed steps
    are the same step indices (and remaps) as the device-timed region."""
    import torch
    host_f0 = torch.from_numpy(f0).pin_memory()
    outs = {k: torch.empty(rc.nx, dtype=torch.float64).pin_memory() for k in ("M", "a", "da", "d2a")}
    se = V.Solver(V.Config.from_run(rc, prec))
    se.sync()

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    V._check(se.L.vm_set_f(se.h, ptr(host_f0), 0), "vm_set_f")
    V._check(se.L.vm_sync(se.h), "vm_sync")
    t_up = time.perf_counter() - t0
    V._check(se.L.vm_step(se.h, args.warmup), "vm_step")
    V._check(se.L.vm_sync(se.h), "vm_sync")
    t1 = time.perf_counter()
    for _ in range(args.steps):
        V._check(se.L.vm_step(se.h, 1), "vm_step")
        V._check(se.L.vm_density_force(se.h, ptr(outs["M"]), ptr(outs["a"]), ptr(outs["da"]),
                                       ptr(outs["d2a"]), 0), "vm_density_force")
    torch.cuda.synchronize(dev)
    t_steps = time.perf_counter() - t1
    te = max_ranks(t_up + t_steps)
    barrier()
    del se
    return {"value": world * rc.nx * rc.nv * args.steps / te, "unit": "cell-updates/s",
            "h2d_bytes_per_step": f0.nbytes / args.steps, "d2h_bytes_per_step": 4 * rc.nx * 8,
            "upload_ms": t_up * 1e3, "steps_ms": t_steps * 1e3,
            "what": f"vm_set_f from pinned host f0 (timed), {args.warmup} untimed steps, then steps "
                    f"{args.warmup}..{args.warmup + args.steps - 1} each with vm_density_force to host (timed)"}


def recon_tiles_ab(V, rc, f0_dev, args, row_stats) -> dict:
    """The FP32-mixed step with the reconstruction in tiles staged by bulk
    copies (recon_mode 1) over the same steps, beside the one-block-per-row
    kernel of the headline: step time and the reconstruction's launch time
    (events around each launch, on a second solve over the same step
    indices, as for the headline)."""
    import torch
    cfg = V.Config.from_run(rc, V.VM_FP32_MIXED)
    cfg.recon_mode = 1
    s = V.Solver(cfg)
    s.set_f(f0_dev)
    s.step(args.warmup)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(args.steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del s
    s = V.Solver(cfg)
    s.set_f(f0_dev)
    s.step(args.warmup)
    s.profile(True)
    s.step(args.steps)
    st = s.profile_read()
    s.profile(False)
    s.sync()
    del s
    rec = st.get("reconstruct", (1, float("nan")))
    row = row_stats.get("reconstruct", (1, float("nan")))
    return {"ms_per_step": ms / args.steps, "value": rc.nx * rc.nv * args.steps / (ms / 1e3),
            "reconstruct_ms": rec[1] / rec[0], "row_kernel_reconstruct_ms": row[1] / row[0],
            "what": "FP32-mixed step with recon_mode 1 (tiles, f_ini patch by cp.async.bulk), same steps"}


def whole_run(V, rc, prec, f0_dev, steps, dev):
    """All `steps` steps of one solve from vm_set_f (remaps included), timed
    with CUDA events on the solver's stream, plus the rate of the last
    tenth of the run (the map's cost grows as the flow shears and mass
    leaves the box)."""
    import torch
    s = V.Solver(V.Config.from_run(rc, prec))
    s.set_f(f0_dev)
    s.sync()
    late = max(1, steps // 10)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(s.stream)
    s.step(steps - late)
    ev[1].record(s.stream)
    s.step(late)
    ev[2].record(s.stream)
    torch.cuda.synchronize(dev)
    s.sync()
    ms = ev[0].elapsed_time(ev[2])
    ms_late = ev[1].elapsed_time(ev[2])
    cells = rc.nx * rc.nv
    del s
    return {"steps": steps, "remaps": steps // rc.n_s, "ms": ms, "value": cells * steps / (ms / 1e3),
            "late_steps": late, "late_value": cells * late / (ms_late / 1e3), "unit": "cell-updates/s",
            "what": f"steps 0..{steps - 1} from vm_set_f, CUDA events on the solver's stream"}


def run_native(args, rank: int, world: int, dist):
    import torch
    from paper_1705_03750_gb300 import vlamet as V

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rc = rank_workload(rank)
    f0 = I.initial_f(rc)
    f0_dev = torch.from_numpy(f0).to(dev)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gpu_id = str(dev.index)
    peaks, peak_kind = _peaks()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_ranks(x: float) -> float:
        return max_over_ranks(x, dist, dev)

    # An idle GPU ran its first tenth of a second or so measurably slower
    # (clock and power state): --spin seconds (default two) of
    # untimed steps of a throwaway solve come before any warm-up or timing.
    if args.spin > 0:
        spin = V.Solver(V.Config.from_run(rc, V.VM_FP32_MIXED))
        spin.set_f(f0_dev)
        t_spin = time.perf_counter() + args.spin
        while time.perf_counter() < t_spin:
            spin.step(20)
            spin.sync()
        del spin
        torch.cuda.synchronize(dev)

    out = {}
    for name, prec in (("fp32", V.VM_FP32_MIXED), ("fp64", V.VM_FP64)):
        if args.precision not in ("both", name):
            continue
        # clock samples during the timed region (the sampler starts first)
        clocks = ClockSampler(gpu_id, f"{args.clock_log}_{name}.csv" if args.clock_log else None).start()
        s = V.Solver(V.Config.from_run(rc, prec))
        s.set_f(f0_dev)
        s.step(args.warmup)
        s.sync()
        stream = s.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = s.launches
        barrier()
        torch.cuda.synchronize(dev)
        clocks.mark_begin()
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clocks.mark_end()
        clocks.stop()
        barrier()
        s.sync()
        ms = max_ranks(e0.elapsed_time(e1))
        launches = s.launches - launches0
        # per-kernel device time over the same step indices (a new solve from
        # f0, the same untimed warm-up; events on the solver's stream around
        # each launch)
        del s
        s = V.Solver(V.Config.from_run(rc, prec))
        s.set_f(f0_dev)
        s.step(args.warmup)
        s.profile(True)
        s.step(args.steps)
        stats = s.profile_read()
        s.profile(False)
        s.sync()
        # end to end through the C ABI with host buffers, over the same step
        # indices as the device-timed region: a new solve uploads f0 from
        # pinned host memory (timed), runs the same untimed warm-up, then
        # every timed step reads the density and force back to the host
        e2e = None
        if not args.no_e2e:
            e2e = e2e_run(V, rc, prec, f0, args, dev, barrier, max_ranks, world)
        # the whole run of the configuration (C2: 1000 steps), device-timed
        whole = None
        if args.whole_run > 0 and not (name == "fp64" and args.whole_run_fp32_only):
            whole = whole_run(V, rc, prec, f0_dev, args.whole_run, dev)
        out[name] = {"ms": ms, "launches": launches, "stats": stats, "clocks": clocks.summary(), "e2e": e2e,
                     "ne": s.ne, "fp32": prec == V.VM_FP32_MIXED, "whole": whole}
        del s
        torch.cuda.synchronize(dev)

    if rank != 0:
        return None
    head = out.get("fp32") or out.get("fp64")
    K = args.steps
    cells = rc.nx * rc.nv
    value = replica_rate(world, cells, K, head["ms"])
    # dominant kernel and its roofline
    stats = head["stats"]
    dom = max(stats, key=lambda k: stats[k][1])
    nl, tms = stats[dom]
    avg_s = tms / nl / 1e3
    alg = algorithmic(dom, rc, head["fp32"], head["ne"])
    roof = {"kernel": dom, "launches_per_step": nl / K, "avg_ms": tms / nl,
            "share_of_step": tms / sum(v[1] for v in stats.values())}
    if alg is not None:
        b, units, per = alg
        ach = b / avg_s / 1e9
        roof.update({"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / peaks["hbm_gbs"], "traffic": ncu_traffic(dom), "per_unit": per,
                     "units": units, "peak_kind": peak_kind})
    # the limiter the counters show for the map and the reconstruction
    iss = issue_roofline(dom, avg_s, (head["clocks"] or {}).get("sm_mhz"))
    if iss is not None:
        roof["issue"] = iss
    # the whole step against the same peak (algorithmic bytes per cell update)
    bpu = step_bytes_per_update(rc, head["fp32"])
    step_ach = bpu * cells * K / (head["ms"] / 1e3) / 1e9
    roof["step"] = {"bytes_per_update": bpu, "achieved": step_ach, "frac": step_ach / peaks["hbm_gbs"]}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": head["ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64 (f32 f/eta/interpolation, f64 elements, map decisions, mass scan)" if head["fp32"] else "f64",
        "data": "synthetic (seeded 16-halo initial condition)",
        "config": {"workload": rc.name, "nx": rc.nx, "nv": rc.nv, "elem_stride": rc.s, "dt": rc.dt,
                   "n_s": rc.n_s, "G": rc.G, "remaps_in_timed_steps": (args.warmup + K) // rc.n_s - args.warmup // rc.n_s,
                   "l2": "working set > L2 (129 MB): no flush", "parallelism": f"replicas x{world}"},
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "whole_run": head["whole"],
        "gpu_launches": head["launches"],
        "roofline": roof,
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1])},
    }
    if "fp64" in out and head is not out["fp64"]:
        f64 = out["fp64"]
        line["fp64_path"] = {"value": replica_rate(world, cells, K, f64["ms"]), "ms_per_step": f64["ms"] / K,
                             "gpu_launches": f64["launches"], "clocks": f64["clocks"],
                             "e2e": f64["e2e"], "whole_run": f64["whole"],
                             "top_kernels": {k: round(v[1], 3) for k, v in sorted(f64["stats"].items(), key=lambda kv: -kv[1][1])[:4]}}
        rl = f64["stats"].get("reconstruct")
        if rl and rl[0] > 0:
            line["fp64_path"]["roofline"] = fp64_roofline(cells, rl[1] / rl[0] / 1e3)
    if world == 1 and not args.no_ab:
        line["recon_tiles"] = recon_tiles_ab(V, rc, f0_dev, args, stats)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(rc, f0)
    if world == 1 and not args.no_serve:
        line["serving"] = serve_sample(args)
    if world == 1 and not args.no_4d:
        line["phase4d"] = phase4d_run(args, dev, peaks, clock_mhz=(head["clocks"] or {}).get("sm_mhz"))
    return line


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(rc, f0, transport_steps: int = 3) -> dict:
    """The FP64 oracle (OpenMP over sites, all host cores) on a bounded
    sample of the same workload: `transport_steps` steps and one remap;
    per-step cost = transport + remap / n_s."""
    import oracle.oracle as O
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, 10 ** 9, rc.G)
    o.set_f(f0)
    t0 = time.perf_counter()
    o.step(transport_steps)
    t1 = time.perf_counter()
    o.remap()
    t2 = time.perf_counter()
    per_step = (t1 - t0) / transport_steps + (t2 - t1) / rc.n_s
    return {"value": rc.nx * rc.nv / per_step, "unit": "cell-updates/s", "cores": _cores(), "kind": "oracle",
            "sample": f"{rc.name}: {transport_steps} transport steps + 1 remap timed "
                      f"({t2 - t0:.1f} s); rate = sites / (step + remap/{rc.n_s})"}


def run_reference(args, rank: int):
    if rank != 0:
        return None
    rc = WORKLOAD
    f0 = I.initial_f(rc)
    import oracle.oracle as O
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_f(f0)
    # one timed step of the full grid costs ~1 s on 16 cores: keep the whole
    # run to a few minutes by timing at most `cap` of the K steps
    cap = max(1, min(args.steps, args.ref_cap))
    o.step(min(args.warmup, 3))
    t0 = time.perf_counter()
    o.step(cap)
    dt = time.perf_counter() - t0
    value = rc.nx * rc.nv * cap / dt
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / cap * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 16-halo initial condition)",
        "config": {"workload": rc.name, "nx": rc.nx, "nv": rc.nv, "elem_stride": rc.s, "dt": rc.dt, "n_s": rc.n_s},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": _cores(), "kind": "oracle",
                         "sample": f"{cap} consecutive full-grid steps of {rc.name} (remaps at their cadence)"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------
# other workloads (their own JSON lines; not the headline)
# ---------------------------------------------------------------------------

# FP64 operations per unit of work of the 4D kernels, counted from the code:
# one inverse-map evaluation Q(P) is 208 (dP 4, s_l 4 x 35, y 28, T^-1 s 28,
# dQ 8); a distance d^2 adds 11; the 15-point interpolation with its
# coordinates adds 97 per reconstructed site
FLOP4_D2 = 219
FLOP4_SITE = 305


def phase4d_run(args, dev, peaks, fp64_peak=None, clock_mhz=None) -> dict:
    """The 4D phase-space path (2D space) on its 64^4 halo workload: K steps
    device-timed after the warm-up (remaps at their cadence inside), a
    profiled pass over the same step indices for the kernel shares and the
    roofline of the dominant kernel, an end-to-end pass through the C ABI
    with host buffers, and the FP64 oracle on a bounded sample."""
    import torch
    from paper_1705_03750_gb300 import inputs4d as I4
    from paper_1705_03750_gb300 import vlamet as V
    from paper_1705_03750_gb300 import vlamet4d as V4
    rc = I4.HALOS4D_64
    if args.n4d != rc.n[0]:
        rc = rc.with_(name=f"halos4d-{args.n4d}^4", n=(args.n4d,) * 4)
    K, W = args.steps4d, max(3, args.warmup4d)
    f0 = I4.initial_f4(rc)
    f0_dev = torch.from_numpy(f0).to(dev)
    sites = rc.sites
    s = V4.Solver4D(V4.config(rc))
    s.set_f(f0_dev)
    s.step(W)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = s.launches
    torch.cuda.synchronize(dev)
    e0.record(s.stream)
    s.step(K)
    e1.record(s.stream)
    torch.cuda.synchronize(dev)
    s.sync()
    ms = e0.elapsed_time(e1)
    launches = s.launches - l0
    del s
    # profiled pass over the same step indices
    s = V4.Solver4D(V4.config(rc))
    s.set_f(f0_dev)
    s.step(W)
    s.sync()
    ev0 = s.map_stats()["d2_evals"]
    s.profile(True)
    s.step(K)
    stats = s.profile_read()
    s.profile(False)
    ev1 = s.map_stats()["d2_evals"]
    s.sync()
    del s
    if fp64_peak is None:
        fp64_peak = V.measure_fp64_peak()
    total = sum(v[1] for v in stats.values())
    dom = max(stats, key=lambda k: stats[k][1])
    nl, tms = stats[dom]
    roof = {"kernel": dom, "launches_per_step": nl / K, "avg_ms": tms / nl, "share_of_step": tms / total}
    L4 = 1
    for a in range(4):
        L4 *= 2 * ((rc.n[a] - 1 + 2 * rc.s - 1) // (2 * rc.s)) + 3
    if dom == "percolate":
        # bound by instruction issue (FP32 tests, integer bookkeeping, atomics;
        # FP64 only at open decisions and contested claims): the capture's
        # warp instructions over the launch time against one warp instruction
        # per scheduler per clock
        n_instr = _keyed(NCU4_INSTR, "percolate", PHASE4D_PREFIX_END)
        mhz = clock_mhz or 2070.0
        peak = SCHEDULERS * mhz * 1e6
        ach = n_instr / (tms / nl / 1e3) if n_instr else None
        roof.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "warp-instr/s",
                     "frac": (ach / peak) if ach else None,
                     "traffic": _keyed(NCU4_TRAFFIC, "percolate", PHASE4D_PREFIX_END),
                     "per_unit": "warp instructions of one launch (ncu capture of this source)",
                     "units": n_instr, "clock_mhz": mhz,
                     "peak_kind": "4 schedulers x 152 SMs x the SM clock",
                     "algorithmic_bytes": 4 * sites + (8 * 64 + 4 * 72) * L4,
                     "fp64_exact_distances_per_launch": (ev1 - ev0) / nl})
    elif dom == "reconstruct":
        flop = FLOP4_SITE * sites
        ach = flop / (tms / nl / 1e3) / 1e12
        roof.update({"bound": "alu", "achieved": ach, "peak": fp64_peak / 1e12, "unit": "TFLOP/s (FP64)",
                     "frac": ach / (fp64_peak / 1e12), "per_unit": f"{FLOP4_SITE} FP64 FLOP per site",
                     "units": sites, "peak_kind": "measured in this run (FP64 FMA chains)"})
    # end to end through the C ABI with host buffers over the same step
    # indices: upload of f0 from pinned host memory, then every timed step
    # reads the pixel masses back to the host
    f0_pin = torch.from_numpy(f0).pin_memory()
    M_host = torch.empty((rc.n[0], rc.n[1]), dtype=torch.float64).pin_memory()
    s = V4.Solver4D(V4.config(rc))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.set_f(f0_pin.numpy())
    up = time.perf_counter() - t0
    s.step(W)
    s.sync()
    t1 = time.perf_counter()
    Mh = M_host.numpy()
    for _ in range(K):
        s.step(1)
        V._check(s.L.vm_4d_density_force(s.h, ctypes.c_void_p(Mh.ctypes.data), None, 0), "vm_4d_density_force")
    t2 = time.perf_counter()
    e2e = {"value": sites * K / (up + (t2 - t1)), "unit": "cell-updates/s",
           "h2d_bytes_per_step": f0.nbytes / K, "d2h_bytes_per_step": 8 * rc.n[0] * rc.n[1],
           "what": f"vm_4d_set_f from pinned host f0 (timed), {W} untimed steps, then {K} steps each with "
                   "vm_4d_density_force to host (timed)"}
    del s
    out = {"workload": rc.name, "sites": sites, "elem_stride": rc.s, "elements": None, "dt": rc.dt, "n_s": rc.n_s,
           "G": rc.G, "steps": K, "warmup": W, "remaps_in_timed_steps": (W + K) // rc.n_s - W // rc.n_s,
           "value": sites * K / (ms / 1e3), "unit": "cell-updates/s", "ms_per_step": ms / K, "dtype": "f64",
           "gpu_launches": launches, "e2e": e2e, "roofline": roof,
           "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1])}}
    out["elements"] = L4
    rl = stats.get("reconstruct")
    if rl and rl[0] > 0:
        # the FP64 reconstruction against the FP64 peak measured in this run
        a_r = FLOP4_SITE * sites / (rl[1] / rl[0] / 1e3) / 1e12
        out["reconstruct_roofline"] = {"bound": "alu", "achieved": a_r, "peak": fp64_peak / 1e12,
                                       "unit": "TFLOP/s (FP64)", "frac": a_r / (fp64_peak / 1e12),
                                       "per_unit": f"{FLOP4_SITE} FP64 FLOP per site", "avg_ms": rl[1] / rl[0]}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_4d(rc, f0)
    return out


def cpu_baseline_4d(rc, f0) -> dict:
    """The FP64 4D oracle (serial) on a bounded sample of the same workload:
    one transport reconstruction (map, f, pixel masses, field) of the 64^4
    state at t = 0; rate = sites / that time."""
    import oracle.oracle4d as Q4
    o = Q4.Oracle4D.from_run(rc)
    o.set_f(f0)
    t0 = time.perf_counter()
    o.reconstruct()
    dt = time.perf_counter() - t0
    return {"value": rc.sites / dt, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{rc.name}: one transport reconstruction (map, f, pixel masses, field) timed ({dt:.1f} s)"}


def run_phase4d(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks, _ = _peaks()
    line = phase4d_run(args, dev, peaks)
    line.update({"metric": "cell-updates/s of the 4D phase-space (2D space) path", "n_gpus": 1,
                 "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                 "data": "synthetic (seeded 4-halo 4D initial condition)",
                 "config": {"workload": line["workload"], "l2": "working set > L2 (129 MB): no flush"}})
    return line

def run_precision(args):
    """8192^2 halos: FP32-mixed vs FP64 GPU paths over many steps (f
    difference, mass and energy), and one step of each against the oracle."""
    import torch
    from paper_1705_03750_gb300 import vlamet as V
    rc = I.HALOS_8192
    f0 = I.initial_f(rc)
    dev = torch.device("cuda", 0)
    f0d = torch.from_numpy(f0).to(dev)
    sol = {}
    for name, prec in (("fp32", V.VM_FP32_MIXED), ("fp64", V.VM_FP64)):
        s = V.Solver(V.Config.from_run(rc, prec))
        s.set_f(f0d)
        sol[name] = s
    steps = args.steps
    hist = []
    t_ms = {"fp32": 0.0, "fp64": 0.0}
    for k in range(0, steps, rc.n_s):
        n = min(rc.n_s, steps - k)
        for name, s in sol.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.step(n)
            e1.record(s.stream)
            torch.cuda.synchronize()
            t_ms[name] += e0.elapsed_time(e1)
        a = sol["fp32"].read_f(dtype=np.float32, out=torch.empty((rc.nx, rc.nv), dtype=torch.float32, device=dev))
        b = sol["fp64"].read_f(out=torch.empty((rc.nx, rc.nv), dtype=torch.float64, device=dev))
        diff = float((a.double() - b).abs().max() / b.abs().max())
        d32, d64 = sol["fp32"].diagnostics(), sol["fp64"].diagnostics()
        hist.append({"step": k + n, "f32_vs_f64_max_rel": diff, "mass32": d32["mass"], "mass64": d64["mass"],
                     "energy32": d32["energy"], "energy64": d64["energy"]})
    out = {"workload": rc.name, "steps": steps, "history": hist,
           "cell_updates_per_s": {n: rc.nx * rc.nv * steps / (t / 1e3) for n, t in t_ms.items()}}
    if not args.no_cpu_baseline:
        import oracle.oracle as O
        o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
        o.set_f(f0)
        o.step(1)
        fo = o.last_f()
        for name, prec in (("fp32", V.VM_FP32_MIXED), ("fp64", V.VM_FP64)):
            s = V.Solver(V.Config.from_run(rc, prec))
            s.set_f(f0d)
            s.step(1)
            out[f"{name}_vs_oracle_step1_max_rel"] = float(np.abs(s.read_f() - fo).max() / np.abs(fo).max())
            dg = s.density_force()
            do = o.density_force()
            out[f"{name}_vs_oracle_step1_mass_rel"] = abs(dg["M"].sum() - do["M"].sum()) / do["M"].sum()
    return out


def run_batch(args):
    """Many uneven independent solves: one graph launch per step (Batch)
    against the plain path (each solve's vm_step on one stream)."""
    import torch
    from paper_1705_03750_gb300 import vlamet as V
    n = args.batch
    cfgs = [I.batch_member(i) for i in range(n)]
    cells = sum(rc.nx * rc.nv for rc in cfgs)
    prec = V.VM_FP32_MIXED
    f0s = [torch.from_numpy(I.initial_f(rc)).cuda() for rc in cfgs]
    stream = torch.cuda.current_stream()

    def fresh():
        ss = [V.Solver(V.Config.from_run(rc, prec), stream=stream) for rc in cfgs]
        for s, f in zip(ss, f0s):
            s.set_f(f)
        return ss
    res = {"workload": f"batch{n}-uneven-64..1024", "solves": n, "sites": cells, "steps": args.steps}
    ss = fresh()
    b = V.Batch(ss, stream=stream)
    tuning = b.autotune(1) if args.autotune else b.tuning()
    b.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res["graph"] = {"cell_updates_per_s": cells * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                    "graph_nodes_per_step": b.launches_per_step(False),
                    "graph_nodes_per_remap_step": b.launches_per_step(True), "tuning": tuning}
    b.close()
    del ss
    # plain path: every solve stepped by its own vm_step call, one stream
    ss = fresh()
    for s in ss:
        s.step(args.warmup)
    torch.cuda.synchronize()
    k = max(1, min(args.steps, 20))
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(k):
        for s in ss:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res["plain"] = {"cell_updates_per_s": cells * k / (ms / 1e3), "ms_per_step": ms / k, "steps_timed": k,
                    "host_s": time.perf_counter() - t0}
    return res


def run_batch_classes(args):
    """Group launches against the same solves stepped one by one (one stream),
    for uniform batches of halo solves: 16 of 1024^2, 64 of 256^2, 256 of
    64^2 (elements every 8 sites above 128, else 4), 20 steps each."""
    import torch
    from paper_1705_03750_gb300 import vlamet as V
    out = {"workload": "uniform halo batches", "steps": args.steps, "classes": {}}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for side, n in ((1024, 16), (256, 64), (64, 256)):
        cfgs = [I.HALOS_4096.with_(nx=side, nv=side, s=8 if side > 128 else 4, seed=i) for i in range(n)]
        f0s = [torch.from_numpy(I.initial_f(rc)).cuda() for rc in cfgs]

        def fresh():
            ss = [V.Solver(V.Config.from_run(rc, V.VM_FP32_MIXED), stream=stream) for rc in cfgs]
            for s_, f in zip(ss, f0s):
                s_.set_f(f)
            return ss

        def timed(fn):
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        ss = fresh()
        b = V.Batch(ss, stream=stream)
        b.step(args.warmup)
        g = timed(lambda: b.step(args.steps))
        b.close()
        ss = fresh()
        for s_ in ss:
            s_.step(args.warmup)

        def plain():
            for _ in range(args.steps):
                for s_ in ss:
                    s_.step(1)
        p = timed(plain)
        sites = side * side * n * args.steps
        out["classes"][f"{n}x{side}^2"] = {"group_cell_updates_per_s": sites / (g / 1e3),
                                          "one_by_one_cell_updates_per_s": sites / (p / 1e3),
                                          "group_ms_per_step": g / args.steps, "one_by_one_ms_per_step": p / args.steps}
        del ss
    return out


def serve_sample(args) -> dict:
    """A reduced serving run for the headline line, on the library's serving
    loop (vm_server_*): 24 seeded halo requests (sides 256-1024, multiples of
    32; 100-400 steps; FP32-mixed; a 150 GB budget, 32 slots; every request
    also remaps when its map's E_map exceeds --emap element spacings), all at
    t = 0 for the saturated throughput, then open-loop Poisson arrivals at 0.5
    and 0.9 of it; p50/p99 latency from arrival to the poll that returns the
    result, and aggregate cell-updates/s."""
    import torch
    from paper_1705_03750_gb300 import vlamet as V
    from paper_1705_03750_gb300.serve import poisson_requests, run_open_loop

    def make(i, nx, nv):
        return I.HALOS_4096.with_(name=f"req{i}", nx=nx, nv=nv, seed=10_000 + i)
    kw = dict(seed=args.seed, make_config=make, sides=(256, 1024), steps=(100, 400))
    ics = {}

    def ic(rc):
        key = (rc.name, rc.nx, rc.nv)
        if key not in ics:
            ics[key] = I.initial_f(rc)
        return ics[key]

    def one(rate):
        reqs = poisson_requests(24, rate=rate, **kw)
        for r in reqs:
            ic(r.config)                # initial conditions prepared before the clock starts
        srv = V.NativeServer(150 << 30, max_active=32, steps_per_tick=args.tick, emap_remap=args.emap)
        rep = run_open_loop(srv, reqs, ic_fn=ic)
        torch.cuda.synchronize()
        srv.close()
        keep = ("requests", "failed", "wall_s", "cell_updates_per_s", "p50_latency_s", "p99_latency_s",
                "peak_active", "group_steps")
        return {k: rep[k] for k in keep}
    sat = one(0.0)
    rate = sat["requests"] / sat["wall_s"]
    out = {"workload": "serve-halos-256..1024 x24, 100-400 steps (vm_server_*)", "emap_remap": args.emap,
           "saturation": {**sat, "requests_per_s": rate}, "rates": []}
    for frac in (0.5, 0.9):
        out["rates"].append({"fraction_of_saturation": frac, "rate_per_s": frac * rate, **one(frac * rate)})
    return out


def run_serve(args):
    """Open-loop Poisson arrivals of seeded halo solves on the library's
    serving loop under a device-memory budget; p50/p99 latency and
    throughput at fractions of saturation."""
    import torch
    from paper_1705_03750_gb300 import vlamet as V
    from paper_1705_03750_gb300.serve import poisson_requests, run_open_loop
    budget = int(args.budget_gb * (1 << 30))

    def make(i, nx, nv):
        return I.HALOS_4096.with_(name=f"req{i}", nx=nx, nv=nv, seed=10_000 + i)
    # seeded per request id and grid: the rate runs draw their arrival times
    # from the same stream, so the same id can come with another grid size
    ics = {}

    def ic(rc):
        key = (rc.name, rc.nx, rc.nv)
        if key not in ics:
            ics[key] = I.initial_f(rc)
        return ics[key]

    def one(reqs):
        for r in reqs:
            ic(r.config)                # initial conditions prepared before the clock starts
        srv = V.NativeServer(budget, max_active=args.max_active, steps_per_tick=args.tick, emap_remap=args.emap)
        rep = run_open_loop(srv, reqs, ic_fn=ic)
        torch.cuda.synchronize()
        srv.close()
        return rep
    base = poisson_requests(args.requests, rate=0.0, seed=args.seed, make_config=make,
                            steps=(args.min_steps, args.max_steps))
    sat = one(base)
    print(json.dumps({"partial_saturation": sat}), file=sys.stderr, flush=True)
    sat_rate = sat["requests"] / sat["wall_s"]
    out = {"workload": "serve-halos-256..2048 (vm_server_*)", "requests": args.requests, "budget_gb": args.budget_gb,
           "emap_remap": args.emap,
           "saturation": {**sat, "requests_per_s": sat_rate}, "rates": []}
    for frac in (0.25, 0.5, 0.75, 0.9, 1.1):
        reqs = poisson_requests(args.requests, rate=frac * sat_rate, seed=args.seed, make_config=make,
                                steps=(args.min_steps, args.max_steps))
        rep = one(reqs)
        out["rates"].append({"fraction_of_saturation": frac, "rate_per_s": frac * sat_rate, **rep})
        print(json.dumps({"partial": out["rates"][-1]}), file=sys.stderr, flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp32", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the reduced serving sample")
    ap.add_argument("--no-ab", action="store_true", help="skip the staged-tile reconstruction comparison")
    ap.add_argument("--whole-run", type=int, default=1000,
                    help="steps of the whole-run rate (the configuration's 1000; 0: skip)")
    ap.add_argument("--whole-run-fp32-only", action="store_true")
    ap.add_argument("--ref-cap", type=int, default=20)
    ap.add_argument("--workload", default="halos4096",
                    choices=["halos4096", "precision8192", "batch", "batch-classes", "serve", "phase4d"])
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--streams", type=int, default=0, help="(unused: one launch per phase for the batch)")
    ap.add_argument("--autotune", type=int, default=1, help="tune the batch's launch shapes on its first steps")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--min-steps", type=int, default=200)
    ap.add_argument("--max-steps", type=int, default=2000)
    ap.add_argument("--tick", type=int, default=5)
    ap.add_argument("--max-active", type=int, default=32)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--emap", type=float, default=0.5,
                    help="serving runs: each request also remaps when its map's E_map exceeds this many "
                         "element spacings (0: every n_s steps only)")
    ap.add_argument("--no-4d", action="store_true", help="skip the 4D phase-space sample")
    ap.add_argument("--steps4d", type=int, default=20, help="timed steps of the 4D phase-space sample")
    ap.add_argument("--warmup4d", type=int, default=3)
    ap.add_argument("--n4d", type=int, default=64, help="nodes per axis of the 4D sample (64: its workload)")
    ap.add_argument("--spin", type=float, default=2.0, help="seconds of untimed steps before the warm-up")
    ap.add_argument("--clock-log", default=None, help="path prefix for the raw clock samples (CSV) of each timed region")
    args = ap.parse_args()
    if args.workload != "halos4096":
        from paper_1705_03750_gb300 import build as B
        B.build()
        fn = {"precision8192": run_precision, "batch": run_batch, "batch-classes": run_batch_classes,
              "serve": run_serve, "phase4d": run_phase4d}[args.workload]
        print(json.dumps(fn(args)))
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as D
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            D.init_process_group("nccl")
            dist = D
        from paper_1705_03750_gb300 import build as B
        B.build()
        line = run_native(args, rank, world, dist)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
