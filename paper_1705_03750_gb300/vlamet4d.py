"""Thin ctypes binding of the 4D phase-space solver (include/vlamet4d.h).

Argument marshalling only: every step runs in the library's CUDA kernels;
PyTorch provides the device workspace and the stream.  There is no fallback:
without the library or a GPU, constructing a Solver4D raises.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import vlamet as V


class Vm4dConfig(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 4), ("lo", C.c_double * 4), ("hi", C.c_double * 4),
        ("elem_stride", C.c_int32), ("dt", C.c_double), ("n_s", C.c_int32), ("G", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("pad", C.c_int32),
        ("max_hole_rounds", C.c_int32),
    ]


class Vm4dDiag(C.Structure):
    _fields_ = [("mass", C.c_double), ("ekin", C.c_double), ("epot", C.c_double),
                ("detT_min", C.c_double), ("detT_max", C.c_double)]


def config(rc, alpha=math.sqrt(3.0) / 4.0, beta=0.5 * (1.0 - math.sqrt(3.0) / 2.0), pad=0,
           max_hole_rounds=0) -> Vm4dConfig:
    """vm_4d_config of a 4D run configuration (grid, box, stride, dt, n_s, G)."""
    return Vm4dConfig((C.c_int32 * 4)(*rc.n), (C.c_double * 4)(*rc.lo), (C.c_double * 4)(*rc.hi),
                      rc.s, rc.dt, rc.n_s, rc.G, alpha, beta, pad, max_hole_rounds)


def workspace_bytes(cfg: Vm4dConfig) -> int:
    return int(V.load().vm_4d_workspace_bytes(C.byref(cfg)))


class Solver4D:
    """One 4D phase-space solve on the current CUDA device, on a torch stream."""

    def __init__(self, cfg: Vm4dConfig, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver4D needs a CUDA device")
        self.L = V.load()
        self.cfg = cfg
        nbytes = workspace_bytes(cfg)
        if nbytes == 0:
            raise ValueError("invalid 4D solver configuration")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) & ~255
        h = C.c_void_p()
        V._check(self.L.vm_4d_create(C.byref(cfg), C.c_void_p(aligned), nbytes,
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h)), "vm_4d_create")
        self.h = h
        Ld = (C.c_int32 * 4)()
        self.ne = int(self.L.vm_4d_num_elements(self.h, Ld))
        self.Ldims = tuple(int(v) for v in Ld)
        self.n = tuple(int(v) for v in cfg.n)

    def close(self):
        if getattr(self, "h", None):
            self.L.vm_4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arg(self, x, shape, dtype: str):
        """(pointer, on_device) of an array a call reads or writes whole; shape,
        type, layout and device are checked (the C ABI takes bare pointers)."""
        shape = tuple(shape)
        if isinstance(x, np.ndarray):
            if x.shape != shape or x.dtype != np.dtype(dtype) or not x.flags.c_contiguous:
                raise ValueError(f"expected a C-contiguous {dtype} array of shape {shape}, got {x.dtype} {x.shape}")
            return C.c_void_p(x.ctypes.data), 0
        import torch
        tdt = {"float64": torch.float64, "int32": torch.int32}[dtype]
        if tuple(x.shape) != shape or x.dtype != tdt or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {dtype} tensor of shape {shape}")
        if x.is_cuda and x.device != self.device:
            raise ValueError(f"tensor on {x.device}, solver on {self.device}")
        return C.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0)

    @property
    def launches(self) -> int:
        return int(self.L.vm_4d_launches(self.h))

    def set_f(self, f0) -> None:
        if isinstance(f0, np.ndarray):
            f0 = np.ascontiguousarray(f0, dtype=np.float64)
        p, dev = self._arg(f0, self.n, "float64")
        V._check(self.L.vm_4d_set_f(self.h, p, dev), "vm_4d_set_f")

    def step(self, k: int = 1) -> None:
        V._check(self.L.vm_4d_step(self.h, int(k)), "vm_4d_step")

    def reconstruct(self) -> None:
        V._check(self.L.vm_4d_reconstruct(self.h), "vm_4d_reconstruct")

    def remap(self) -> None:
        V._check(self.L.vm_4d_remap(self.h), "vm_4d_remap")

    def map_stats(self) -> dict:
        out = (C.c_int32 * 3)()
        ev = C.c_int64()
        V._check(self.L.vm_4d_map_stats(self.h, out, C.byref(ev)), "vm_4d_map_stats")
        return {"window_overflows": int(out[0]), "holes": int(out[1]), "rounds": int(out[2]),
                "d2_evals": int(ev.value)}

    def profile(self, on: bool) -> None:
        V._check(self.L.vm_4d_profile(self.h, int(bool(on))), "vm_4d_profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, ms)} since the last read (synchronises)."""
        n = 32
        la = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        k = int(self.L.vm_4d_profile_read(self.h, la, ms, n))
        out = {}
        for i in range(min(k, n)):
            if la[i]:
                out[self.L.vm_4d_kernel_name(i).decode()] = (int(la[i]), float(ms[i]))
        return out

    def sync(self) -> None:
        V._check(self.L.vm_4d_sync(self.h), "vm_4d_sync")

    def _read(self, fn, shape, dtype, out=None):
        if out is None:
            out = np.empty(shape, dtype=dtype)
        p, dev = self._arg(out, shape, np.dtype(dtype).name)
        V._check(getattr(self.L, fn)(self.h, p, dev), fn)
        return out

    def read_f(self, out=None):
        return self._read("vm_4d_read_f", self.n, np.float64, out)

    def read_fini(self, out=None):
        return self._read("vm_4d_read_fini", self.n, np.float64, out)

    def read_eta(self, out=None):
        return self._read("vm_4d_read_eta", self.n, np.float64, out)

    def read_map(self, out=None):
        return self._read("vm_4d_read_map", self.n, np.int32, out)

    def elements(self) -> np.ndarray:
        return self._read("vm_4d_get_elements", (self.ne, 60), np.float64)

    def set_elements(self, el) -> None:
        if isinstance(el, np.ndarray):
            el = np.ascontiguousarray(el, dtype=np.float64)
        p, dev = self._arg(el, (self.ne, 60), "float64")
        V._check(self.L.vm_4d_set_elements(self.h, p, dev), "vm_4d_set_elements")

    def diagnostics(self) -> dict:
        d = Vm4dDiag()
        V._check(self.L.vm_4d_diagnostics(self.h, C.byref(d)), "vm_4d_diagnostics")
        return {k: getattr(d, k) for k, _ in Vm4dDiag._fields_}

    def density_force(self) -> dict:
        M = np.empty(self.n[:2])
        F = np.empty(self.n[:2] + (12,))
        V._check(self.L.vm_4d_density_force(self.h, C.c_void_p(M.ctypes.data), C.c_void_p(F.ctypes.data), 0),
                 "vm_4d_density_force")
        return {"M": M, "field": F}
