"""Seeded synthetic initial conditions for the 4D phase-space (2D space) solver.

Workloads only (grids, boxes, time steps, seeded phase-space distributions):
none of the solver's arithmetic, and nothing else from the package is
imported, so the CUDA path and the FP64 oracle can both be fed from it.

The paper implements the 2D phase-space case and names the 4D one as the
next step (Sec. 5); it gives no 4D test.  The workload here carries its 2D
halo test over: a sum of warm Gaussian halos, isotropic in space and in
velocity, with centres, widths and masses drawn from the seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class RunConfig4D:
    """One 4D solve: nodes and box per axis (x, y, vx, vy), element stride,
    time step, remap period, G (lap phi = 4 pi G rho in 2D space)."""
    name: str
    n: tuple
    lo: tuple
    hi: tuple
    s: int
    dt: float
    n_s: int
    G: float
    steps: int
    halos: int = 4
    seed: int = 0

    @property
    def d(self) -> tuple:
        return tuple((self.hi[a] - self.lo[a]) / (self.n[a] - 1) for a in range(4))

    def axis(self, a: int) -> np.ndarray:
        return self.lo[a] + np.arange(self.n[a], dtype=np.float64) * self.d[a]

    @property
    def sites(self) -> int:
        return int(np.prod(self.n))

    def with_(self, **kw) -> "RunConfig4D":
        return replace(self, **kw)


def draw_halos4d(seed: int, n: int) -> dict:
    """Halo parameters in a fixed draw order: centres (x, y) ~ U[-0.4, 0.4],
    mean velocities ~ U[-0.3, 0.3], sigma_x log-uniform [0.12, 0.25],
    sigma_v log-uniform [0.15, 0.3], masses log-uniform [0.1, 1] normalised
    to a total of 1."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(-0.4, 0.4, size=(n, 2))
    cv = rng.uniform(-0.3, 0.3, size=(n, 2))
    sx = np.exp(rng.uniform(math.log(0.12), math.log(0.25), size=n))
    sv = np.exp(rng.uniform(math.log(0.15), math.log(0.3), size=n))
    m = np.exp(rng.uniform(math.log(0.1), math.log(1.0), size=n))
    m = m / m.sum()
    return {"cx": cx, "cv": cv, "sx": sx, "sv": sv, "m": m}


def halos4d(cfg: RunConfig4D) -> np.ndarray:
    """f = sum_k m_k / ((2 pi)^2 sx_k^2 sv_k^2)
           exp(-|r - r_k|^2 / (2 sx_k^2) - |v - v_k|^2 / (2 sv_k^2)),
    on the nodes, f[i0, i1, i2, i3] (vy fastest), FP64."""
    h = draw_halos4d(cfg.seed, cfg.halos)
    x, y, u, w = (cfg.axis(a) for a in range(4))
    f = np.zeros(cfg.n)
    for k in range(cfg.halos):
        ex = np.exp(-0.5 * ((x - h["cx"][k, 0]) / h["sx"][k]) ** 2)
        ey = np.exp(-0.5 * ((y - h["cx"][k, 1]) / h["sx"][k]) ** 2)
        eu = np.exp(-0.5 * ((u - h["cv"][k, 0]) / h["sv"][k]) ** 2)
        ew = np.exp(-0.5 * ((w - h["cv"][k, 1]) / h["sv"][k]) ** 2)
        amp = h["m"][k] / ((2.0 * math.pi) ** 2 * h["sx"][k] ** 2 * h["sv"][k] ** 2)
        f += amp * np.einsum("i,j,k,l->ijkl", ex, ey, eu, ew)
    return f


def initial_f4(cfg: RunConfig4D) -> np.ndarray:
    return halos4d(cfg)


BOX_LO = (-1.0, -1.0, -1.5, -1.5)
BOX_HI = (1.0, 1.0, 1.5, 1.5)
# the measured workload: 64^4 = 16.8 M sites, elements every 4 sites
HALOS4D_64 = RunConfig4D("halos4d-64^4", (64, 64, 64, 64), BOX_LO, BOX_HI, 4, 0.005, 10, 1.0, 100)
# parity cases the oracle finishes in seconds: a cube and a ragged shape
HALOS4D_16 = HALOS4D_64.with_(name="halos4d-16^4", n=(16, 16, 16, 16), n_s=4, steps=8)
HALOS4D_RAGGED = HALOS4D_64.with_(name="halos4d-18x14x20x12", n=(18, 14, 20, 12), n_s=4, steps=8,
                                  seed=3)
FREE4D_16 = HALOS4D_16.with_(name="free4d-16^4-G0", G=0.0)
WORKLOADS4D = {c.name: c for c in (HALOS4D_64, HALOS4D_16, HALOS4D_RAGGED, FREE4D_16)}
