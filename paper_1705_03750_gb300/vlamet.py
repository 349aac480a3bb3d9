"""Thin ctypes binding of libvlamet (the C ABI declared in include/vlamet.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device workspace and the stream.  There
is no fallback: if the library is missing or no GPU is present, constructing
a Solver raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvlamet.so")

VM_FP64, VM_FP32_MIXED = 0, 1
VM_DTYPE_F64, VM_DTYPE_F32 = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "workspace too small", 3: "CUDA runtime error",
          4: "unexplored-site repair did not converge", 5: "influence region larger than the largest window",
          6: "memory budget exceeded", 7: "call out of order", 8: "internal consistency check failed",
          9: "checkpoint file could not be written or read"}

# Names of every entry point declared in include/vlamet.h.
EXPORTS = ["vm_config_default", "vm_workspace_bytes", "vm_create", "vm_destroy", "vm_status_string",
           "vm_lattice", "vm_set_f", "vm_set_elements", "vm_get_elements", "vm_compute_map",
           "vm_reconstruct", "vm_step", "vm_remap", "vm_density_force", "vm_read_f", "vm_read_fini",
           "vm_read_eta", "vm_read_map", "vm_diagnostics", "vm_sync", "vm_launch_count",
           "vm_profile", "vm_profile_read", "vm_force_from_f_static",
           "vm_batch_create", "vm_batch_step", "vm_batch_launches_per_step", "vm_batch_destroy",
           "vm_batch_autotune", "vm_batch_tuning",
           "vm_server_pool_bytes", "vm_server_create", "vm_server_submit", "vm_server_poll", "vm_server_result",
           "vm_server_stats", "vm_server_destroy",
           "vm_last_cuda_error", "vm_cuda_error_name", "vm_save", "vm_load", "vm_measure_fp64_peak",
           # include/vlamet4d.h
           "vm_4d_workspace_bytes", "vm_4d_create", "vm_4d_destroy", "vm_4d_set_f", "vm_4d_step",
           "vm_4d_reconstruct", "vm_4d_remap", "vm_4d_read_f", "vm_4d_read_fini", "vm_4d_read_eta",
           "vm_4d_read_map", "vm_4d_density_force", "vm_4d_get_elements", "vm_4d_set_elements",
           "vm_4d_num_elements", "vm_4d_launches", "vm_4d_map_stats", "vm_4d_sync",
           "vm_4d_profile", "vm_4d_profile_read", "vm_4d_kernel_name", "vm_4d_diagnostics"]

VM_STATIC_FORCE_MAX_NX = 16384


class VmConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("nv", C.c_int32),
        ("x_lo", C.c_double), ("x_hi", C.c_double), ("v_lo", C.c_double), ("v_hi", C.c_double),
        ("elem_stride", C.c_int32), ("dt", C.c_double), ("n_s", C.c_int32), ("G", C.c_double),
        ("precision", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double),
        ("pad", C.c_int32), ("literal_fd", C.c_int32), ("max_hole_rounds", C.c_int32),
        ("map_windows", C.c_int32), ("emap_remap", C.c_double), ("c_dyn", C.c_double),
        ("f_th", C.c_double), ("recon_mode", C.c_int32),
    ]


class VmDiag(C.Structure):
    _fields_ = [("mass", C.c_double), ("energy", C.c_double), ("detT_min", C.c_double),
                ("detT_max", C.c_double), ("step", C.c_int64), ("cycle", C.c_int32),
                ("holes", C.c_int32), ("hole_rounds", C.c_int32), ("overflow_elements", C.c_int32),
                ("tier1_more", C.c_int32), ("last_tier_elements", C.c_int32),
                ("exact_tests", C.c_int32), ("bad_where", C.c_int32), ("entropy", C.c_double),
                ("l1", C.c_double), ("l2", C.c_double), ("emap", C.c_double), ("emap_remaps", C.c_int64),
                ("time", C.c_double), ("last_dt", C.c_double),
                ("lattice_range", C.c_int32 * 4), ("site_rect", C.c_int32 * 4)]


class VmServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_active", C.c_int32), ("steps_per_tick", C.c_int32),
                ("precision", C.c_int32)]


class VmServerDone(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("finish_s", C.c_double)]


class VmServerStat(C.Structure):
    _fields_ = [("waiting", C.c_int32), ("active", C.c_int32), ("finished", C.c_int32), ("peak_active", C.c_int32),
                ("used_bytes", C.c_int64), ("peak_bytes", C.c_int64), ("ticks", C.c_int64),
                ("group_steps", C.c_int64), ("remap_groups", C.c_int64)]


class VmKernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class VlametError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Open libvlamet.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libvlamet.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    sig = {
        "vm_config_default": (None, [C.POINTER(VmConfig)]),
        "vm_workspace_bytes": (C.c_size_t, [C.POINTER(VmConfig)]),
        "vm_create": (i32, [C.POINTER(VmConfig), vp, C.c_size_t, vp, C.POINTER(vp)]),
        "vm_destroy": (None, [vp]),
        "vm_status_string": (C.c_char_p, [i32]),
        "vm_lattice": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "vm_set_f": (i32, [vp, vp, i32]),
        "vm_set_elements": (i32, [vp, vp, i32]),
        "vm_get_elements": (i32, [vp, vp, i32]),
        "vm_compute_map": (i32, [vp]),
        "vm_reconstruct": (i32, [vp]),
        "vm_step": (i32, [vp, i32]),
        "vm_remap": (i32, [vp]),
        "vm_density_force": (i32, [vp, vp, vp, vp, vp, i32]),
        "vm_read_f": (i32, [vp, vp, i32, i32]),
        "vm_read_fini": (i32, [vp, vp, i32, i32]),
        "vm_read_eta": (i32, [vp, vp, i32, i32]),
        "vm_read_map": (i32, [vp, vp, i32]),
        "vm_diagnostics": (i32, [vp, C.POINTER(VmDiag)]),
        "vm_sync": (i32, [vp]),
        "vm_launch_count": (i64, [vp]),
        "vm_profile": (i32, [vp, i32]),
        "vm_profile_read": (i32, [vp, C.POINTER(VmKernelStat), i32]),
        "vm_force_from_f_static": (i32, [vp, i32, i32, i32, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, i32, vp, vp, vp, vp, vp]),
        "vm_batch_create": (i32, [C.POINTER(vp), i32, i32, vp, C.POINTER(vp)]),
        "vm_batch_step": (i32, [vp, i32]),
        "vm_batch_launches_per_step": (i64, [vp, i32]),
        "vm_batch_destroy": (None, [vp]),
        "vm_batch_autotune": (i32, [vp, i32]),
        "vm_server_pool_bytes": (C.c_size_t, [C.POINTER(VmServerConfig)]),
        "vm_server_create": (i32, [C.POINTER(VmServerConfig), vp, C.c_size_t, vp, C.POINTER(vp)]),
        "vm_server_submit": (i32, [vp, C.POINTER(VmConfig), vp, i32, C.POINTER(i64)]),
        "vm_server_poll": (i32, [vp, C.POINTER(VmServerDone), i32, C.POINTER(i32)]),
        "vm_server_result": (i32, [vp, i64, vp, vp, vp, vp]),
        "vm_server_stats": (i32, [vp, C.POINTER(VmServerStat)]),
        "vm_server_destroy": (None, [vp]),
        "vm_batch_tuning": (i32, [vp, C.POINTER(i32), dp]),
        "vm_last_cuda_error": (i32, []),
        "vm_cuda_error_name": (C.c_char_p, [i32]),
        "vm_save": (i32, [vp, C.c_char_p]),
        "vm_load": (i32, [vp, C.c_char_p]),
        "vm_measure_fp64_peak": (i32, [i32, vp, dp]),
        "vm_4d_workspace_bytes": (C.c_size_t, [vp]),
        "vm_4d_create": (i32, [vp, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "vm_4d_destroy": (None, [vp]),
        "vm_4d_set_f": (i32, [vp, vp, i32]),
        "vm_4d_step": (i32, [vp, i32]),
        "vm_4d_reconstruct": (i32, [vp]),
        "vm_4d_remap": (i32, [vp]),
        "vm_4d_read_f": (i32, [vp, vp, i32]),
        "vm_4d_read_fini": (i32, [vp, vp, i32]),
        "vm_4d_read_eta": (i32, [vp, vp, i32]),
        "vm_4d_read_map": (i32, [vp, vp, i32]),
        "vm_4d_density_force": (i32, [vp, vp, vp, i32]),
        "vm_4d_get_elements": (i32, [vp, vp, i32]),
        "vm_4d_set_elements": (i32, [vp, vp, i32]),
        "vm_4d_num_elements": (i32, [vp, C.POINTER(i32)]),
        "vm_4d_launches": (i64, [vp]),
        "vm_4d_map_stats": (i32, [vp, C.POINTER(i32), C.POINTER(i64)]),
        "vm_4d_profile": (i32, [vp, i32]),
        "vm_4d_profile_read": (i32, [vp, C.POINTER(i64), dp, i32]),
        "vm_4d_kernel_name": (C.c_char_p, [i32]),
        "vm_4d_diagnostics": (i32, [vp, vp]),
        "vm_4d_sync": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str) -> None:
    if st != 0:
        if st == 3:
            L = load()
            code = int(L.vm_last_cuda_error())
            name = L.vm_cuda_error_name(code)
            where = f"{where} [{name.decode() if name else code}]"
        raise VlametError(st, where)


@dataclass
class Config:
    nx: int
    nv: int
    x_lo: float
    x_hi: float
    v_lo: float
    v_hi: float
    s: int
    dt: float
    n_s: int
    G: float
    precision: int = VM_FP64
    alpha: float = math.sqrt(3.0) / 4.0
    beta: float = 0.5 * (1.0 - math.sqrt(3.0) / 2.0)
    pad: int = 0
    literal_fd: int = 0
    max_hole_rounds: int = 0
    map_windows: int = 0
    emap_remap: float = 0.0
    c_dyn: float = 0.0
    f_th: float = 0.0
    recon_mode: int = 0

    @classmethod
    def from_run(cls, rc, precision: int = VM_FP64) -> "Config":
        return cls(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G, precision)

    def c(self) -> VmConfig:
        return VmConfig(self.nx, self.nv, self.x_lo, self.x_hi, self.v_lo, self.v_hi, self.s, self.dt,
                        self.n_s, self.G, self.precision, self.alpha, self.beta, self.pad, self.literal_fd,
                        self.max_hole_rounds, self.map_windows, self.emap_remap, self.c_dyn, self.f_th,
                        self.recon_mode)


def workspace_bytes(cfg: Config) -> int:
    c = cfg.c()
    return int(load().vm_workspace_bytes(C.byref(c)))


def force_from_f_static(f, cfg: Config, out: dict, stream=None) -> None:
    """Pixel masses and force of a device tensor f ([nx, nv], float64 or
    float32) into the device tensors out["a"], out["da"], out["d2a"] (and
    out["M"] if present), through the allocation-free entry point: its only
    scratch is a static device array of at most VM_STATIC_FORCE_MAX_NX pixel
    masses shared by all calls (serialise calls that could overlap)."""
    import torch
    L = load()
    if cfg.nx > VM_STATIC_FORCE_MAX_NX:
        raise ValueError(f"nx = {cfg.nx} exceeds the static scratch limit of {VM_STATIC_FORCE_MAX_NX} pixels")
    assert f.is_cuda and f.is_contiguous() and tuple(f.shape) == (cfg.nx, cfg.nv)
    dtype = {torch.float64: VM_DTYPE_F64, torch.float32: VM_DTYPE_F32}[f.dtype]
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    for k, t in out.items():
        if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float64 and tuple(t.shape) == (cfg.nx,)):
            raise ValueError(f"out[{k!r}] must be a contiguous float64 device tensor of shape ({cfg.nx},)")
    ptr = lambda k: C.c_void_p(out[k].data_ptr()) if k in out else None  # noqa: E731
    _check(L.vm_force_from_f_static(C.c_void_p(f.data_ptr()), dtype, cfg.nx, cfg.nv, cfg.x_lo, cfg.x_hi,
                                    cfg.v_lo, cfg.v_hi, cfg.G, cfg.literal_fd, ptr("M"), ptr("a"), ptr("da"),
                                    ptr("d2a"), C.c_void_p(st.cuda_stream)), "vm_force_from_f_static")


def measure_fp64_peak(iters: int = 20000, stream=None) -> float:
    """FP64 FLOP/s of the current device from the library's FMA-chain probe
    (vm_measure_fp64_peak); synchronises."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    r = C.c_double()
    _check(load().vm_measure_fp64_peak(int(iters), C.c_void_p(st.cuda_stream), C.byref(r)),
           "vm_measure_fp64_peak")
    return r.value


class Solver:
    """One solve on the current CUDA device, on a torch stream."""

    def __init__(self, cfg: Config, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device")
        self.L = load()
        self.cfg = cfg
        self._c = cfg.c()
        nbytes = int(self.L.vm_workspace_bytes(C.byref(self._c)))
        if nbytes == 0:
            raise ValueError("invalid solver configuration")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p()
        _check(self.L.vm_create(C.byref(self._c), C.c_void_p(aligned), nbytes,
                                C.c_void_p(self.stream.cuda_stream), C.byref(h)), "vm_create")
        self.h = h
        ne, lx, lv = C.c_int32(), C.c_int32(), C.c_int32()
        self.L.vm_lattice(self.h, C.byref(ne), C.byref(lx), C.byref(lv))
        self.ne, self.Lx, self.Lv = ne.value, lx.value, lv.value
        self.nx, self.nv = cfg.nx, cfg.nv
        self.fp32 = cfg.precision == VM_FP32_MIXED

    def close(self):
        if getattr(self, "h", None):
            self.L.vm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- pointers: a torch tensor (device) or a numpy array (host) ----
    @staticmethod
    def _ptr(x):
        if isinstance(x, np.ndarray):
            assert x.flags.c_contiguous
            return C.c_void_p(x.ctypes.data), 0
        assert x.is_contiguous()
        return C.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0)

    def _arg(self, x, shape, dtype: str):
        """(pointer, on_device) of an array that a call reads or writes whole.
        The C ABI takes bare pointers, so the shape, element type, layout and
        device are checked here: a smaller buffer would be read past its end."""
        shape = tuple(shape)
        if isinstance(x, np.ndarray):
            if x.shape != shape or x.dtype != np.dtype(dtype) or not x.flags.c_contiguous:
                raise ValueError(f"expected a C-contiguous {dtype} array of shape {shape}, "
                                 f"got {x.dtype} {x.shape}")
            return C.c_void_p(x.ctypes.data), 0
        import torch
        tdt = {"float64": torch.float64, "float32": torch.float32, "int32": torch.int32}[dtype]
        if tuple(x.shape) != shape or x.dtype != tdt or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {dtype} tensor of shape {shape}, got {x.dtype} {tuple(x.shape)}")
        if x.is_cuda and x.device != self.device:
            raise ValueError(f"tensor on {x.device}, solver on {self.device}")
        return C.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0)

    def set_f(self, f0) -> None:
        if isinstance(f0, np.ndarray):
            f0 = np.ascontiguousarray(f0, dtype=np.float64)
        p, dev = self._arg(f0, (self.nx, self.nv), "float64")
        _check(self.L.vm_set_f(self.h, p, dev), "vm_set_f")

    def set_elements(self, soa12) -> None:
        if isinstance(soa12, np.ndarray):
            soa12 = np.ascontiguousarray(soa12, dtype=np.float64)
        p, dev = self._arg(soa12, (12, self.ne), "float64")
        _check(self.L.vm_set_elements(self.h, p, dev), "vm_set_elements")

    def elements(self) -> np.ndarray:
        out = np.empty((12, self.ne))
        _check(self.L.vm_get_elements(self.h, C.c_void_p(out.ctypes.data), 0), "vm_get_elements")
        return out

    def compute_map(self) -> None:
        _check(self.L.vm_compute_map(self.h), "vm_compute_map")

    def reconstruct(self) -> None:
        _check(self.L.vm_reconstruct(self.h), "vm_reconstruct")

    def step(self, n: int = 1) -> None:
        _check(self.L.vm_step(self.h, int(n)), "vm_step")

    def remap(self) -> None:
        _check(self.L.vm_remap(self.h), "vm_remap")

    def sync(self) -> None:
        _check(self.L.vm_sync(self.h), "vm_sync")

    def save(self, path) -> None:
        """Checkpoint of the state carried between steps (see vm_save)."""
        _check(self.L.vm_save(self.h, os.fsencode(path)), "vm_save")

    def load(self, path) -> None:
        """Replace this solver's state by a checkpoint of the same run (vm_load)."""
        _check(self.L.vm_load(self.h, os.fsencode(path)), "vm_load")

    def density_force(self, out=None) -> dict:
        """M, a, a', a'' ([nx] float64 each) of the last reconstruction.  With
        ``out`` (a dict of device tensors) the copy stays on the device."""
        if out is not None:
            ptrs = []
            for k in ("M", "a", "da", "d2a"):
                if k in out:
                    p, dev = self._arg(out[k], (self.nx,), "float64")
                    if not dev:
                        raise ValueError("out tensors must be on the device")
                    ptrs.append(p)
                else:
                    ptrs.append(None)
            _check(self.L.vm_density_force(self.h, *ptrs, 1), "vm_density_force")
            return out
        res = {k: np.empty(self.nx) for k in ("M", "a", "da", "d2a")}
        _check(self.L.vm_density_force(self.h, *(C.c_void_p(res[k].ctypes.data) for k in ("M", "a", "da", "d2a")), 0),
               "vm_density_force")
        return res

    def _read(self, fn, name, dtype=np.float64, out=None):
        code = VM_DTYPE_F64 if dtype == np.float64 else VM_DTYPE_F32
        if out is not None:
            p, dev = self._arg(out, (self.nx, self.nv), "float64" if code == VM_DTYPE_F64 else "float32")
            _check(fn(self.h, p, code, dev), name)
            return out
        res = np.empty((self.nx, self.nv), dtype=dtype)
        _check(fn(self.h, C.c_void_p(res.ctypes.data), code, 0), name)
        return res

    def read_f(self, dtype=np.float64, out=None):
        return self._read(self.L.vm_read_f, "vm_read_f", dtype, out)

    def read_fini(self, dtype=np.float64, out=None):
        return self._read(self.L.vm_read_fini, "vm_read_fini", dtype, out)

    def read_eta(self, dtype=np.float64, out=None):
        return self._read(self.L.vm_read_eta, "vm_read_eta", dtype, out)

    def read_map(self) -> np.ndarray:
        res = np.empty((self.nx, self.nv), dtype=np.int32)
        _check(self.L.vm_read_map(self.h, C.c_void_p(res.ctypes.data), 0), "vm_read_map")
        return res

    def diagnostics(self) -> dict:
        d = VmDiag()
        _check(self.L.vm_diagnostics(self.h, C.byref(d)), "vm_diagnostics")
        out = {k: getattr(d, k) for k, _ in VmDiag._fields_}
        for k in ("lattice_range", "site_rect"):
            out[k] = tuple(int(x) for x in out[k])
        return out

    def profile(self, enable: bool = True) -> None:
        """Start (or stop) per-kernel event timing; resets the totals."""
        _check(self.L.vm_profile(self.h, int(enable)), "vm_profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since profile()."""
        buf = (VmKernelStat * 32)()
        n = self.L.vm_profile_read(self.h, buf, 32)
        if n < 0:
            raise VlametError(1, "vm_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 32))}

    @property
    def launches(self) -> int:
        return int(self.L.vm_launch_count(self.h))


class Batch:
    """Many independent solves advanced together: every phase of a step is
    one launch for the whole batch, the step one CUDA graph launch.  All
    solvers must have had set_f, share their precision and remap phase.
    ``nstreams`` is not used (kept for compatibility)."""

    def __init__(self, solvers, nstreams: int = 0, stream=None):
        import torch
        self.L = load()
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        arr = (C.c_void_p * len(self.solvers))(*[s.h for s in self.solvers])
        h = C.c_void_p()
        _check(self.L.vm_batch_create(arr, len(self.solvers), int(nstreams), C.c_void_p(self.stream.cuda_stream),
                                      C.byref(h)), "vm_batch_create")
        self.h = h

    def step(self, n: int = 1) -> None:
        _check(self.L.vm_batch_step(self.h, int(n)), "vm_batch_step")

    def launches_per_step(self, with_remap: bool = False) -> int:
        return int(self.L.vm_batch_launches_per_step(self.h, int(with_remap)))

    def autotune(self, trials: int = 1) -> dict:
        """Tune the persistent blocks of each phase on real steps (4 x trials
        transport steps are taken); returns the chosen shape."""
        _check(self.L.vm_batch_autotune(self.h, int(trials)), "vm_batch_autotune")
        return self.tuning()

    def tuning(self) -> dict:
        bps = (C.c_int32 * 5)()
        ms = (C.c_double * 5)()
        tuned = self.L.vm_batch_tuning(self.h, bps, ms)
        names = ("drift_taylor", "map", "reconstruct", "scan_force", "kick_drift")
        return {"tuned": bool(tuned), "blocks_per_sm": dict(zip(names, list(bps))),
                "ms_per_step": dict(zip(names, list(ms)))}

    def close(self):
        if getattr(self, "h", None):
            self.L.vm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NativeServer:
    """The library's serving loop (vm_server_*): continuous batching of
    submitted solves on one device pool.  ``budget_bytes`` of the pool hold
    the solves' workspaces; ``poll()`` drives it without waiting for the
    device and returns the requests finished since the last call.
    ``emap_remap`` (> 0) is every request's E_map remap threshold unless
    submit() gives its own."""

    def __init__(self, budget_bytes: int, max_active: int = 32, steps_per_tick: int = 5,
                 precision: int = VM_FP32_MIXED, stream=None, device=None, emap_remap: float = 0.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("NativeServer needs a CUDA device")
        self.L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.precision = precision
        self.emap_remap = float(emap_remap)
        self._c = VmServerConfig(int(budget_bytes), int(max_active), int(steps_per_tick), int(precision))
        reserve = int(self.L.vm_server_pool_bytes(C.byref(self._c)))
        nbytes = reserve + int(budget_bytes)
        self._pool = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = (self._pool.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        _check(self.L.vm_server_create(C.byref(self._c), C.c_void_p(base), nbytes, C.c_void_p(self.stream.cuda_stream),
                                       C.byref(h)), "vm_server_create")
        self.h = h
        self.nx = {}
        self._done = (VmServerDone * 256)()

    def submit(self, rc, f0: np.ndarray, steps: int, emap_remap: float | None = None) -> int:
        c = Config.from_run(rc, self.precision)
        c.emap_remap = self.emap_remap if emap_remap is None else float(emap_remap)
        cfg = c.c()
        f0 = np.ascontiguousarray(f0, dtype=np.float64)
        if f0.shape != (rc.nx, rc.nv):
            raise ValueError(f"f0 must have shape ({rc.nx}, {rc.nv})")
        rid = C.c_int64()
        _check(self.L.vm_server_submit(self.h, C.byref(cfg), C.c_void_p(f0.ctypes.data), int(steps), C.byref(rid)),
               "vm_server_submit")
        self.nx[rid.value] = rc.nx
        return rid.value

    def poll(self) -> list:
        n = C.c_int32()
        _check(self.L.vm_server_poll(self.h, self._done, len(self._done), C.byref(n)), "vm_server_poll")
        return [{"id": d.id, "status": d.status, "submit_s": d.submit_s, "admit_s": d.admit_s,
                 "finish_s": d.finish_s} for d in self._done[:n.value]]

    def result(self, rid: int) -> dict:
        nx = self.nx[rid]
        out = {k: np.empty(nx) for k in ("M", "a", "da", "d2a")}
        _check(self.L.vm_server_result(self.h, int(rid), *[C.c_void_p(out[k].ctypes.data) for k in ("M", "a", "da", "d2a")]),
               "vm_server_result")
        return out

    def stats(self) -> dict:
        st = VmServerStat()
        _check(self.L.vm_server_stats(self.h, C.byref(st)), "vm_server_stats")
        return {k: getattr(st, k) for k, _ in VmServerStat._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.vm_server_destroy(self.h)
            self.h = None
        self._pool = None           # the device pool goes back with the handle

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
