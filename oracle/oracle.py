"""ctypes wrapper of the FP64 C oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The oracle is plain serial C (``vlamet_oracle.c``), optionally built with
OpenMP over independent sites (the paper's own parallelisation, Sec. 3.1);
both builds give bit-identical results because no floating-point reduction
crosses threads.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlamet_oracle.c")
_SRC4 = os.path.join(_HERE, "vlamet4d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[bool, C.CDLL] = {}


def build(openmp: bool = True, force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add) and return the path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libvlamet_oracle_omp.so" if openmp else "libvlamet_oracle.so")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC4),
                                             os.path.getmtime(os.path.join(_HERE, "vlamet_oracle.h")),
                                             os.path.getmtime(os.path.join(_HERE, "vlamet4d_oracle.h")))):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unknown-pragmas", _SRC, _SRC4, "-o", out + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class VoConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("nv", C.c_int32),
        ("x_lo", C.c_double), ("x_hi", C.c_double), ("v_lo", C.c_double), ("v_hi", C.c_double),
        ("s", C.c_int32), ("dt", C.c_double), ("n_s", C.c_int32), ("G", C.c_double),
        ("alpha", C.c_double), ("beta", C.c_double), ("pad", C.c_int32),
        ("literal_fd", C.c_int32), ("max_hole_rounds", C.c_int32),
    ]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def lib(openmp: bool = True) -> C.CDLL:
    with _lock:
        if openmp in _libs:
            return _libs[openmp]
        L = C.CDLL(build(openmp))
        sig = {
            "vo_qinterp": (C.c_double, [_D, C.c_int32, C.c_int32, C.c_double, C.c_double]),
            "vo_spline_solve_1d": (None, [C.c_int32, _D, _D]),
            "vo_spline_solve_2d": (None, [C.c_int32, C.c_int32, _D, _D]),
            "vo_bspline3": (C.c_double, [C.c_double]),
            "vo_spline_eval": (C.c_double, [_D, C.c_int32, C.c_int32, C.c_double, C.c_double]),
            "vo_taylor_one": (None, [_D, C.c_double, C.c_double, _D]),
            "vo_qofp": (None, [_D, C.c_double, C.c_double, _D, _D]),
            "vo_W": (C.c_double, [C.c_double]),
            "vo_force_from_mass": (None, [_D, C.c_int32, C.c_double, C.c_double, C.c_int32, _D, _D, _D]),
            "vo_tsc": (C.c_double, [_D, C.c_int32, C.c_double, C.c_double, C.c_double]),
            "vo_alpha_offsets": (C.c_int32, [C.c_double, C.c_double, C.c_double, _I32]),
            "vo_beta_offsets": (C.c_int32, [C.c_double, C.c_double, C.c_double, _I32]),
            "vo_create": (C.c_void_p, [C.POINTER(VoConfig)]),
            "vo_destroy": (None, [C.c_void_p]),
            "vo_num_elements": (C.c_int32, [C.c_void_p]),
            "vo_lattice_dims": (C.c_int32, [C.c_void_p, _I32, _I32]),
            "vo_set_f": (C.c_int32, [C.c_void_p, _D]),
            "vo_get_elements": (None, [C.c_void_p, _D]),
            "vo_set_elements": (None, [C.c_void_p, _D]),
            "vo_get_taylor": (None, [C.c_void_p, _D]),
            "vo_compute_map": (C.c_int32, [C.c_void_p, _I32]),
            "vo_map_stats": (C.c_int32, [C.c_void_p, _I64, _I64, _I32]),
            "vo_component_bbox": (None, [C.c_void_p, _I32]),
            "vo_reconstruct": (C.c_int32, [C.c_void_p, _D]),
            "vo_density_force": (None, [C.c_void_p, _D, _D, _D, _D, _D]),
            "vo_step": (C.c_int32, [C.c_void_p, C.c_int32]),
            "vo_remap": (C.c_int32, [C.c_void_p]),
            "vo_remap_resample": (C.c_int32, [C.c_void_p, _D, _D]),
            "vo_get_fini": (None, [C.c_void_p, _D]),
            "vo_get_eta": (None, [C.c_void_p, _D]),
            "vo_get_last_f": (None, [C.c_void_p, _D]),
            "vo_step_count": (C.c_int64, [C.c_void_p]),
            "vo_cycle_step": (C.c_int32, [C.c_void_p]),
            "vo_diagnostics": (None, [C.c_void_p, _D, _D, _D, _D]),
            "vo_casimirs": (None, [C.c_void_p, _D, _D, _D]),
            "vo_emap": (C.c_double, [C.c_void_p]),
            "vo_set_cdyn": (None, [C.c_void_p, C.c_double]),
            "vo_set_fth": (None, [C.c_void_p, C.c_double]),
            "vo_domain": (None, [C.c_void_p, _I32, _I32]),
            "vo_time": (C.c_double, [C.c_void_p]),
            "vo_last_dt": (C.c_double, [C.c_void_p]),
            "vo_push_frozen": (None, [C.c_void_p, _D, _D, _D, C.c_double, C.c_double, C.c_int32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _libs[openmp] = L
        return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I32)


ALPHA = math.sqrt(3.0) / 4.0
BETA = 0.5 * (1.0 - math.sqrt(3.0) / 2.0)


# ---- low-level pieces -------------------------------------------------------

def qinterp(F: np.ndarray, u: float, w: float) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().vo_qinterp(_dp(F), F.shape[0], F.shape[1], float(u), float(w))


def spline_solve_1d(f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().vo_spline_solve_1d(f.size, _dp(f), _dp(out))
    return out


def spline_solve_2d(f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().vo_spline_solve_2d(f.shape[0], f.shape[1], _dp(f), _dp(out))
    return out


def bspline3(t: float) -> float:
    return lib().vo_bspline3(float(t))


def spline_eval(eta: np.ndarray, u: float, w: float) -> float:
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    return lib().vo_spline_eval(_dp(eta), eta.shape[0], eta.shape[1], float(u), float(w))


def taylor_one(el12, Qx: float, Qv: float) -> np.ndarray:
    el = np.ascontiguousarray(el12, dtype=np.float64)
    out = np.empty(14)
    lib().vo_taylor_one(_dp(el), float(Qx), float(Qv), _dp(out))
    return out


def qofp(tay14: np.ndarray, Px: float, Pv: float) -> tuple[float, float]:
    t = np.ascontiguousarray(tay14, dtype=np.float64)
    a, b = C.c_double(), C.c_double()
    lib().vo_qofp(_dp(t), float(Px), float(Pv), C.byref(a), C.byref(b))
    return a.value, b.value


def W(x: float) -> float:
    return lib().vo_W(float(x))


def force_from_mass(M: np.ndarray, dx: float, G: float, literal_fd: bool = False):
    M = np.ascontiguousarray(M, dtype=np.float64)
    a, da, d2a = (np.empty_like(M) for _ in range(3))
    lib().vo_force_from_mass(_dp(M), M.size, float(dx), float(G), int(literal_fd), _dp(a), _dp(da), _dp(d2a))
    return a, da, d2a


def tsc(A: np.ndarray, ext_lo: float, ext_hi: float, u: float) -> float:
    A = np.ascontiguousarray(A, dtype=np.float64)
    return lib().vo_tsc(_dp(A), A.size, float(ext_lo), float(ext_hi), float(u))


def alpha_offsets(xi: float, ze: float, alpha: float = None) -> list:
    ab = np.zeros(18, dtype=np.int32)
    n = lib().vo_alpha_offsets(float(xi), float(ze), ALPHA if alpha is None else float(alpha), _ip(ab))
    return [tuple(ab[2 * q:2 * q + 2]) for q in range(n)]


def beta_offsets(xi: float, ze: float, beta: float = None) -> list:
    ab = np.zeros(18, dtype=np.int32)
    n = lib().vo_beta_offsets(float(xi), float(ze), BETA if beta is None else float(beta), _ip(ab))
    return [tuple(ab[2 * q:2 * q + 2]) for q in range(n)]


# ---- solver -----------------------------------------------------------------

class Oracle:
    """The whole method on one grid (one solve), FP64, on the host."""

    def __init__(self, nx, nv, x_lo, x_hi, v_lo, v_hi, s, dt, n_s, G,
                 alpha=ALPHA, beta=BETA, pad=None, literal_fd=False, max_hole_rounds=0,
                 openmp=True):
        self.cfg = VoConfig(nx, nv, x_lo, x_hi, v_lo, v_hi, s, dt, n_s, G, alpha, beta,
                            s if pad is None else pad, int(literal_fd), max_hole_rounds)
        self.L = lib(openmp)
        self.h = self.L.vo_create(C.byref(self.cfg))
        if not self.h:
            raise ValueError("invalid oracle configuration")
        self.nx, self.nv = nx, nv
        lx, lv = C.c_int32(), C.c_int32()
        self.ne = self.L.vo_lattice_dims(self.h, C.byref(lx), C.byref(lv))
        self.Lx, self.Lv = lx.value, lv.value
        self.dx = (x_hi - x_lo) / (nx - 1)
        self.dv = (v_hi - v_lo) / (nv - 1)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.vo_destroy(h)
            self.h = None

    def set_f(self, f0: np.ndarray) -> None:
        f0 = np.ascontiguousarray(f0, dtype=np.float64).reshape(self.nx, self.nv)
        self.L.vo_set_f(self.h, _dp(f0))

    def elements(self) -> np.ndarray:
        out = np.empty((self.ne, 12))
        self.L.vo_get_elements(self.h, _dp(out))
        return out

    def set_elements(self, el: np.ndarray) -> None:
        el = np.ascontiguousarray(el, dtype=np.float64).reshape(self.ne, 12)
        self.L.vo_set_elements(self.h, _dp(el))

    def taylor(self) -> np.ndarray:
        out = np.empty((self.ne, 14))
        self.L.vo_get_taylor(self.h, _dp(out))
        return out

    def compute_map(self) -> tuple[np.ndarray, int]:
        out = np.empty((self.nx, self.nv), dtype=np.int32)
        st = self.L.vo_compute_map(self.h, _ip(out))
        return out, st

    def map_stats(self) -> dict:
        a, b, c = C.c_int64(), C.c_int64(), C.c_int32()
        self.L.vo_map_stats(self.h, C.byref(a), C.byref(b), C.byref(c))
        return {"multi_claims": a.value, "holes": b.value, "rounds": c.value}

    def component_bbox(self) -> np.ndarray:
        """[ne, 4]: i_min, i_max, j_min, j_max of each element's component in
        the last percolation (min > max when empty)."""
        out = np.empty((self.ne, 4), dtype=np.int32)
        self.L.vo_component_bbox(self.h, _ip(out))
        return out

    def reconstruct(self) -> np.ndarray:
        out = np.empty((self.nx, self.nv))
        st = self.L.vo_reconstruct(self.h, _dp(out))
        if st != 0:
            raise RuntimeError(f"oracle map did not converge (status {st})")
        return out

    def density_force(self) -> dict:
        M, a, da, d2a = (np.empty(self.nx) for _ in range(4))
        mt = C.c_double()
        self.L.vo_density_force(self.h, _dp(M), _dp(a), _dp(da), _dp(d2a), C.byref(mt))
        return {"M": M, "a": a, "da": da, "d2a": d2a, "Mtot": mt.value}

    def step(self, n: int = 1) -> int:
        return self.L.vo_step(self.h, int(n))

    def remap(self) -> int:
        return self.L.vo_remap(self.h)

    def remap_resample(self) -> tuple[np.ndarray, np.ndarray]:
        f = np.empty((self.nx, self.nv))
        q = np.empty((self.nx, self.nv, 2))
        self.L.vo_remap_resample(self.h, _dp(f), _dp(q))
        return f, q

    def fini(self) -> np.ndarray:
        out = np.empty((self.nx, self.nv))
        self.L.vo_get_fini(self.h, _dp(out))
        return out

    def eta(self) -> np.ndarray:
        out = np.empty((self.nx, self.nv))
        self.L.vo_get_eta(self.h, _dp(out))
        return out

    def last_f(self) -> np.ndarray:
        out = np.empty((self.nx, self.nv))
        self.L.vo_get_last_f(self.h, _dp(out))
        return out

    @property
    def step_count(self) -> int:
        return self.L.vo_step_count(self.h)

    @property
    def cycle_step(self) -> int:
        return self.L.vo_cycle_step(self.h)

    def diagnostics(self) -> dict:
        m, e, lo, hi = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        self.L.vo_diagnostics(self.h, C.byref(m), C.byref(e), C.byref(lo), C.byref(hi))
        se, l1, l2 = C.c_double(), C.c_double(), C.c_double()
        self.L.vo_casimirs(self.h, C.byref(se), C.byref(l1), C.byref(l2))
        return {"mass": m.value, "energy": e.value, "detT_min": lo.value, "detT_max": hi.value,
                "entropy": se.value, "l1": l1.value, "l2": l2.value, "emap": self.L.vo_emap(self.h)}

    def set_cdyn(self, c_dyn: float) -> None:
        """Variable time step min(dt, c_dyn / sqrt(rho_max)) (0: constant)."""
        self.L.vo_set_cdyn(self.h, float(c_dyn))

    def set_fth(self, f_th: float) -> None:
        """Adaptive computing domain (Sec. 2.2.1, eq. constrf; Sec. 2.3) with
        threshold f_th (0: the fixed box); takes effect at the next set_f or
        remap."""
        self.L.vo_set_fth(self.h, float(f_th))

    def domain(self) -> dict:
        """Existing lattice range (klo, khi, llo, lhi) and the last map's site
        rectangle (i_lo, i_hi, j_lo, j_hi)."""
        a = np.zeros(4, dtype=np.int32)
        r = np.zeros(4, dtype=np.int32)
        self.L.vo_domain(self.h, _ip(a), _ip(r))
        return {"lattice": tuple(int(x) for x in a), "rect": tuple(int(x) for x in r)}

    def time(self) -> float:
        return self.L.vo_time(self.h)

    def last_dt(self) -> float:
        return self.L.vo_last_dt(self.h)

    def push_frozen(self, a, da, d2a, ext_lo, ext_hi, nsteps):
        a, da, d2a = (np.ascontiguousarray(z, dtype=np.float64) for z in (a, da, d2a))
        self.L.vo_push_frozen(self.h, _dp(a), _dp(da), _dp(d2a), float(ext_lo), float(ext_hi), int(nsteps))
