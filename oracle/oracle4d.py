"""ctypes wrapper of the FP64 C oracle of the 4D phase-space step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU-baseline leg of
``bench.py``.  The product path never imports it.  The C code
(``vlamet4d_oracle.c``) is compiled into the same library as the 2D oracle.
"""
from __future__ import annotations

import ctypes as C
import math
import threading

import numpy as np

from . import oracle as O

ALPHA = math.sqrt(3.0) / 4.0
BETA = 0.5 * (1.0 - math.sqrt(3.0) / 2.0)

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_lock = threading.Lock()
_done: set = set()


class Vo4Config(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 4), ("lo", C.c_double * 4), ("hi", C.c_double * 4),
        ("s", C.c_int32), ("dt", C.c_double), ("n_s", C.c_int32), ("G", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("pad", C.c_int32),
        ("max_hole_rounds", C.c_int32),
    ]


def lib(openmp: bool = False) -> C.CDLL:
    L = O.lib(openmp)
    with _lock:
        if openmp in _done:
            return L
        sig = {
            "vo4_qinterp": (C.c_double, [_D, _I32, _D]),
            "vo4_spline_solve": (None, [_I32, _D, _D]),
            "vo4_spline_eval": (C.c_double, [_D, _I32, _D]),
            "vo4_taylor_one": (None, [_D, _D, _D]),
            "vo4_qofp": (None, [_D, _D, _D]),
            "vo4_alpha_offsets": (C.c_int32, [_D, C.c_double, _I32]),
            "vo4_beta_offsets": (C.c_int32, [_D, C.c_double, _I32]),
            "vo4_field_at_node": (None, [_D, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                         C.c_double, C.c_int64, C.c_int64, _D]),
            "vo4_accel_at_node": (None, [_D, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                         C.c_double, C.c_int64, C.c_int64, _D]),
            "vo4_create": (C.c_void_p, [C.POINTER(Vo4Config)]),
            "vo4_destroy": (None, [C.c_void_p]),
            "vo4_num_elements": (C.c_int32, [C.c_void_p]),
            "vo4_lattice_dims": (None, [C.c_void_p, _I32]),
            "vo4_set_f": (C.c_int32, [C.c_void_p, _D]),
            "vo4_get_elements": (None, [C.c_void_p, _D]),
            "vo4_set_elements": (None, [C.c_void_p, _D]),
            "vo4_get_taylor": (None, [C.c_void_p, _D]),
            "vo4_compute_map": (C.c_int32, [C.c_void_p, _I32]),
            "vo4_get_map": (None, [C.c_void_p, _I32]),
            "vo4_map_stats": (None, [C.c_void_p, _I64, _I64, _I32]),
            "vo4_reconstruct": (C.c_int32, [C.c_void_p, _D]),
            "vo4_density_force": (None, [C.c_void_p, _D, _D, _D]),
            "vo4_step": (C.c_int32, [C.c_void_p, C.c_int32]),
            "vo4_remap": (C.c_int32, [C.c_void_p]),
            "vo4_remap_resample": (C.c_int32, [C.c_void_p, _D, _D]),
            "vo4_get_fini": (None, [C.c_void_p, _D]),
            "vo4_get_eta": (None, [C.c_void_p, _D]),
            "vo4_get_last_f": (None, [C.c_void_p, _D]),
            "vo4_step_count": (C.c_int64, [C.c_void_p]),
            "vo4_diagnostics": (None, [C.c_void_p, _D, _D, _D, _D, _D]),
            "vo4_push_frozen": (None, [C.c_void_p, _D, C.c_int32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _done.add(openmp)
        return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


def _n(n) -> np.ndarray:
    return np.ascontiguousarray(n, dtype=np.int32)


def _u(u) -> np.ndarray:
    return np.ascontiguousarray(u, dtype=np.float64)


def qinterp(F: np.ndarray, u) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().vo4_qinterp(_dp(F), _ip(_n(F.shape)), _dp(_u(u)))


def spline_solve(f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    eta = np.empty_like(f)
    lib().vo4_spline_solve(_ip(_n(f.shape)), _dp(f), _dp(eta))
    return eta


def spline_eval(eta: np.ndarray, u) -> float:
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    return lib().vo4_spline_eval(_dp(eta), _ip(_n(eta.shape)), _dp(_u(u)))


def taylor_one(el60, Qm) -> np.ndarray:
    out = np.empty(64)
    lib().vo4_taylor_one(_dp(_u(el60)), _dp(_u(Qm)), _dp(out))
    return out


def qofp(tay64, P) -> np.ndarray:
    out = np.empty(4)
    lib().vo4_qofp(_dp(_u(tay64)), _dp(_u(P)), _dp(out))
    return out


def alpha_offsets(xi, alpha: float = ALPHA) -> list:
    off = np.zeros(4 * 16, dtype=np.int32)
    n = lib().vo4_alpha_offsets(_dp(_u(xi)), float(alpha), _ip(off))
    return [tuple(int(v) for v in off[4 * q:4 * q + 4]) for q in range(n)]


def beta_offsets(xi, beta: float = BETA) -> list:
    off = np.zeros(4 * 81, dtype=np.int32)
    n = lib().vo4_beta_offsets(_dp(_u(xi)), float(beta), _ip(off))
    return [tuple(int(v) for v in off[4 * q:4 * q + 4]) for q in range(n)]


def accel_at_node(M: np.ndarray, dx: float, dy: float, G: float, i: int, j: int) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = np.empty(2)
    lib().vo4_accel_at_node(_dp(M), M.shape[0], M.shape[1], dx, dy, G, i, j, _dp(out))
    return out


def field_at_node(M: np.ndarray, dx: float, dy: float, G: float, i: int, j: int) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = np.empty(12)
    lib().vo4_field_at_node(_dp(M), M.shape[0], M.shape[1], dx, dy, G, i, j, _dp(out))
    return out


class Oracle4D:
    """The whole 4D-phase-space method on one grid, FP64, on the host."""

    def __init__(self, n, lo, hi, s, dt, n_s, G, alpha=ALPHA, beta=BETA, pad=None,
                 max_hole_rounds=0):
        self.n = tuple(int(v) for v in n)
        self.cfg = Vo4Config((C.c_int32 * 4)(*self.n), (C.c_double * 4)(*lo),
                             (C.c_double * 4)(*hi), s, dt, n_s, G, alpha, beta,
                             s if pad is None else pad, max_hole_rounds)
        self.L = lib()
        self.h = self.L.vo4_create(C.byref(self.cfg))
        if not self.h:
            raise ValueError("invalid oracle configuration")
        self.ne = self.L.vo4_num_elements(self.h)
        Ld = np.zeros(4, dtype=np.int32)
        self.L.vo4_lattice_dims(self.h, _ip(Ld))
        self.Ldims = tuple(int(v) for v in Ld)
        self.d = tuple((hi[a] - lo[a]) / (self.n[a] - 1) for a in range(4))
        self.lo, self.hi = tuple(lo), tuple(hi)

    @classmethod
    def from_run(cls, rc, **kw):
        return cls(rc.n, rc.lo, rc.hi, rc.s, rc.dt, rc.n_s, rc.G, **kw)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.vo4_destroy(h)
            self.h = None

    def set_f(self, f0: np.ndarray) -> None:
        f0 = np.ascontiguousarray(f0, dtype=np.float64).reshape(self.n)
        self.L.vo4_set_f(self.h, _dp(f0))

    def elements(self) -> np.ndarray:
        out = np.empty((self.ne, 60))
        self.L.vo4_get_elements(self.h, _dp(out))
        return out

    def set_elements(self, el: np.ndarray) -> None:
        el = np.ascontiguousarray(el, dtype=np.float64).reshape(self.ne, 60)
        self.L.vo4_set_elements(self.h, _dp(el))

    def taylor(self) -> np.ndarray:
        out = np.empty((self.ne, 64))
        self.L.vo4_get_taylor(self.h, _dp(out))
        return out

    def compute_map(self) -> tuple[np.ndarray, int]:
        out = np.empty(self.n, dtype=np.int32)
        st = self.L.vo4_compute_map(self.h, _ip(out))
        return out, st

    def last_map(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        self.L.vo4_get_map(self.h, _ip(out))
        return out

    def map_stats(self) -> dict:
        a, b, c = C.c_int64(), C.c_int64(), C.c_int32()
        self.L.vo4_map_stats(self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"multi_claims": a.value, "holes": b.value, "rounds": c.value}

    def reconstruct(self) -> np.ndarray:
        out = np.empty(self.n)
        st = self.L.vo4_reconstruct(self.h, _dp(out))
        if st:
            raise RuntimeError(f"oracle map status {st}")
        return out

    def density_force(self) -> dict:
        M = np.empty(self.n[:2])
        F = np.empty(self.n[:2] + (12,))
        mt = C.c_double()
        self.L.vo4_density_force(self.h, _dp(M), _dp(F), C.byref(mt))
        return {"M": M, "field": F, "Mtot": mt.value}

    def step(self, k: int = 1) -> int:
        return self.L.vo4_step(self.h, k)

    def remap(self) -> int:
        return self.L.vo4_remap(self.h)

    def remap_resample(self) -> tuple[np.ndarray, np.ndarray]:
        out = np.empty(self.n)
        qr = np.empty(self.n + (4,))
        self.L.vo4_remap_resample(self.h, _dp(out), _dp(qr))
        return out, qr

    def fini(self) -> np.ndarray:
        out = np.empty(self.n)
        self.L.vo4_get_fini(self.h, _dp(out))
        return out

    def eta(self) -> np.ndarray:
        out = np.empty(self.n)
        self.L.vo4_get_eta(self.h, _dp(out))
        return out

    def last_f(self) -> np.ndarray:
        out = np.empty(self.n)
        self.L.vo4_get_last_f(self.h, _dp(out))
        return out

    def step_count(self) -> int:
        return self.L.vo4_step_count(self.h)

    def diagnostics(self) -> dict:
        v = [C.c_double() for _ in range(5)]
        self.L.vo4_diagnostics(self.h, *[C.byref(x) for x in v])
        keys = ("mass", "ekin", "epot", "detT_min", "detT_max")
        return {k: x.value for k, x in zip(keys, v)}

    def push_frozen(self, coef12, nsteps: int) -> None:
        c = np.ascontiguousarray(coef12, dtype=np.float64)
        assert c.shape == (12,)
        self.L.vo4_push_frozen(self.h, _dp(c), nsteps)
