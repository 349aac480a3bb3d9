"""Seeded synthetic initial conditions and run configurations.

This module holds the workloads only (grids, boxes, time steps, seeded
phase-space distributions).  It contains none of the solver's arithmetic and
imports nothing else from the package, so the CUDA path and the FP64 oracle
can both be fed from it.

Workloads, shaped after the paper's tests (Sec. 3.2):
  * isothermal (Spitzer) sheet, the stationary solution used as the paper's
    first test, normalised to total mass 1 with G = 1;
  * a sum of warm Gaussian halos, standing in for the paper's random set of
    stationary clouds (whose exact construction is not given in the paper);
  * a free-streaming (G = 0) run on the Spitzer grid;
  * the paper's truncated Gaussian initial condition (Sec. 3.2, eqs. monfg,
    gauini): rho_G exp(-(x^2 + v^2)/(2 sigma_G^2)) inside radius R, cut
    smoothly beyond it by max[1 + 2 tanh((R - r)/eta_G), 0];
  * the paper's apodised thermal-equilibrium sheet (Sec. 3.2, eqs. apofs,
    apod) in the paper's units (phi'' = 2 rho, i.e. G = 1/(2 pi)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

ALPHA = math.sqrt(3.0) / 4.0            # Sec. 2.3.3, alpha = sqrt(3)/4
BETA = 0.5 * (1.0 - math.sqrt(3.0) / 2.0)  # Sec. 2.3.3, beta = (1 - sqrt(3)/2)/2


@dataclass(frozen=True)
class RunConfig:
    """One solve: grid, box, element stride, time step, remap period, G."""
    name: str
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
    steps: int
    ic: str = "spitzer"          # "spitzer" | "halos"
    ic_params: dict = field(default_factory=dict)
    seed: int = 0

    @property
    def dx(self) -> float:
        return (self.x_hi - self.x_lo) / (self.nx - 1)

    @property
    def dv(self) -> float:
        return (self.v_hi - self.v_lo) / (self.nv - 1)

    def x(self) -> np.ndarray:
        return self.x_lo + np.arange(self.nx, dtype=np.float64) * self.dx

    def v(self) -> np.ndarray:
        return self.v_lo + np.arange(self.nv, dtype=np.float64) * self.dv

    def with_(self, **kw) -> "RunConfig":
        return replace(self, **kw)


# ---- initial conditions ------------------------------------------------------

def spitzer(x: np.ndarray, v: np.ndarray, sigma: float = 0.5, G: float = 1.0,
            mass: float = 1.0) -> np.ndarray:
    """Isothermal sheet f = rho0/(sqrt(2 pi) sigma) sech^2(x/x0) exp(-v^2/2sigma^2).

    For phi'' = 4 pi G rho the self-consistent scale is x0 = sigma^2/(pi G M)
    with rho0 = M/(2 x0); x and v broadcast against each other.
    """
    x0 = sigma * sigma / (math.pi * G * mass) if G != 0 else sigma * sigma / math.pi
    rho0 = mass / (2.0 * x0)
    return (rho0 / (math.sqrt(2.0 * math.pi) * sigma)) / np.cosh(x / x0) ** 2 * \
        np.exp(-0.5 * (v / sigma) ** 2)


@dataclass(frozen=True)
class Halos:
    """Parameters of a sum of Gaussian phase-space halos."""
    xc: np.ndarray
    vc: np.ndarray
    sx: np.ndarray
    sv: np.ndarray
    m: np.ndarray

    def __call__(self, x: np.ndarray, v: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(x, v).shape)
        for k in range(self.m.size):
            out += self.m[k] / (2.0 * math.pi * self.sx[k] * self.sv[k]) * np.exp(
                -0.5 * ((x - self.xc[k]) / self.sx[k]) ** 2 - 0.5 * ((v - self.vc[k]) / self.sv[k]) ** 2)
        return out


    def on_grid(self, x: np.ndarray, v: np.ndarray) -> np.ndarray:
        """The same sum on the tensor grid x (rows) by v (columns), using that
        each halo is a product of a Gaussian in x and one in v."""
        out = np.zeros((x.size, v.size))
        for k in range(self.m.size):
            gx = self.m[k] / (2.0 * math.pi * self.sx[k] * self.sv[k]) * np.exp(-0.5 * ((x - self.xc[k]) / self.sx[k]) ** 2)
            gv = np.exp(-0.5 * ((v - self.vc[k]) / self.sv[k]) ** 2)
            out += np.outer(gx, gv)
        return out


def draw_halos(seed: int, n: int = 16, centre: float = 0.5, sx=(0.02, 0.1), sv=(0.05, 0.2),
               mass=(0.1, 1.0)) -> Halos:
    """Draw halo parameters from numpy's default_rng(seed) in a fixed order:
    x centres, v centres, log sigma_x, log sigma_v, log masses; masses are
    normalised to a total of 1."""
    rng = np.random.default_rng(seed)
    xc = rng.uniform(-centre, centre, n)
    vc = rng.uniform(-centre, centre, n)
    sxs = np.exp(rng.uniform(math.log(sx[0]), math.log(sx[1]), n))
    svs = np.exp(rng.uniform(math.log(sv[0]), math.log(sv[1]), n))
    m = np.exp(rng.uniform(math.log(mass[0]), math.log(mass[1]), n))
    m = m / m.sum()
    return Halos(xc, vc, sxs, svs, m)


def gaussian_ic(x, v, rho=4.0, sigma=0.2, R=1.0, eta=0.02):
    """The paper's Gaussian initial condition (Sec. 3.2): rho exp(-r^2 /
    (2 sigma^2)) for r = sqrt(x^2 + v^2) <= R, times max[1 + 2 tanh((R - r) /
    eta), 0] beyond R.  The paper's values rho = 4, sigma = 0.2, R = 1,
    eta = 0.02 give a total mass close to 1 (a Gaussian cut at 5 sigma)."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    r = np.sqrt(x * x + v * v)
    g = rho * np.exp(-0.5 * (x * x + v * v) / (sigma * sigma))
    cut = np.maximum(1.0 + 2.0 * np.tanh((R - r) / eta), 0.0)
    return np.where(r <= R, g, g * cut)


def apodised_spitzer(x, v, rho=4.0, sigma=0.2, eta=0.02):
    """The paper's thermal-equilibrium sheet (Sec. 3.2, eq. apofs),
    f_S = rho / ch^2(sqrt(sqrt(2 pi) rho / sigma) x) exp(-v^2 / (2 sigma^2)),
    apodised as in eq. apod.  The apodising function is printed as
    g(y) = eta max[1 + 2 th((y - eta)/eta), 0], whose leading eta would scale
    the whole sheet by about 3 eta and contradict the printed maximum
    projected density (about 2, that of f_S itself); it is read like the cut
    of the Gaussian initial condition printed beside it (eq. monfg2):
    f = f_S where f_S >= eta, and f_S max[1 + 2 th((f_S - eta)/eta), 0]
    below, so f is continuous and vanishes where f_S < eta (1 - atanh(1/2)).
    In the paper's units (phi'' = 2 rho) the sheet is stationary."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    k = math.sqrt(math.sqrt(2.0 * math.pi) * rho / sigma)
    fs = rho / np.cosh(k * x) ** 2 * np.exp(-0.5 * (v / sigma) ** 2)
    cut = np.maximum(1.0 + 2.0 * np.tanh((fs - eta) / eta), 0.0)
    return np.where(fs >= eta, fs, fs * cut)


def initial_f(cfg: RunConfig) -> np.ndarray:
    """f0 sampled on the nodes, [nx, nv] float64, v fastest."""
    X, V = np.meshgrid(cfg.x(), cfg.v(), indexing="ij")
    if cfg.ic == "spitzer":
        return spitzer(X, V, sigma=cfg.ic_params.get("sigma", 0.5), G=cfg.G if cfg.G else 1.0)
    if cfg.ic == "halos":
        h = draw_halos(cfg.seed, n=cfg.ic_params.get("n", 16))
        return h.on_grid(cfg.x(), cfg.v())
    if cfg.ic == "gauss":
        return gaussian_ic(X, V, **cfg.ic_params)
    if cfg.ic == "apod":
        return apodised_spitzer(X, V, **cfg.ic_params)
    if cfg.ic == "blob":
        # a single warm Gaussian well inside the box (free-streaming checks)
        p = cfg.ic_params
        return np.exp(-0.5 * ((X - p.get("x0", 0.0)) / p.get("sx", 0.15)) ** 2
                      - 0.5 * ((V - p.get("v0", 0.0)) / p.get("sv", 0.3)) ** 2)
    raise ValueError(cfg.ic)


def ic_function(cfg: RunConfig):
    """The initial condition as a callable f0(x, v) (for exact free streaming)."""
    if cfg.ic == "spitzer":
        sig = cfg.ic_params.get("sigma", 0.5)
        return lambda x, v: spitzer(x, v, sigma=sig, G=cfg.G if cfg.G else 1.0)
    if cfg.ic == "halos":
        return draw_halos(cfg.seed, n=cfg.ic_params.get("n", 16))
    if cfg.ic == "gauss":
        return lambda x, v: gaussian_ic(x, v, **cfg.ic_params)
    if cfg.ic == "apod":
        return lambda x, v: apodised_spitzer(x, v, **cfg.ic_params)
    if cfg.ic == "blob":
        p = cfg.ic_params
        return lambda x, v: np.exp(-0.5 * ((x - p.get("x0", 0.0)) / p.get("sx", 0.15)) ** 2
                                   - 0.5 * ((v - p.get("v0", 0.0)) / p.get("sv", 0.3)) ** 2)
    raise ValueError(cfg.ic)


# ---- the named workloads -----------------------------------------------------

SPITZER_128 = RunConfig("spitzer-128x128-G1", 128, 128, -1.0, 1.0, -2.5, 2.5, 4, 0.005, 20, 1.0, 200,
                        "spitzer", {"sigma": 0.5})
FREE_128 = SPITZER_128.with_(name="free-streaming-128x128-G0", G=0.0)
HALOS_4096 = RunConfig("halos16-4096x4096", 4096, 4096, -1.0, 1.0, -1.5, 1.5, 8, 0.002, 25, 1.0, 1000,
                       "halos", {"n": 16}, seed=0)
HALOS_8192 = HALOS_4096.with_(name="halos16-8192x8192", nx=8192, nv=8192, steps=500)
# the paper's Gaussian run on a box just wider than the cut radius (Delta = 2.4/127)
GAUSS_128 = RunConfig("gauss-128x128-G1", 128, 128, -1.2, 1.2, -1.2, 1.2, 4, 0.005, 20, 1.0, 200,
                      "gauss", {"rho": 4.0, "sigma": 0.2, "R": 1.0, "eta": 0.02})

# the paper's apodised thermal equilibrium (rho_S = 4, sigma_S = 0.2, eta = 0.02)
# in its units (2 pi G = 1), on a box just wider than the apodised support
# (|x| < 0.53, |v| < 0.70); the paper's time step 0.0025 and n_s = 25
APOD_128 = RunConfig("apodised-spitzer-128x128", 128, 128, -0.6, 0.6, -0.8, 0.8, 4, 0.0025, 25,
                     1.0 / (2.0 * math.pi), 200, "apod", {"rho": 4.0, "sigma": 0.2, "eta": 0.02})

WORKLOADS = {c.name: c for c in (SPITZER_128, FREE_128, HALOS_4096, HALOS_8192, GAUSS_128, APOD_128)}


def batch_member(index: int, base_seed: int = 1000) -> RunConfig:
    """One of the many independent solves of the batched workload: sides drawn
    independently from {64, ..., 1024}, a Spitzer sheet (sigma ~ U[0.3, 0.7],
    v box +-5 sigma) or 4-16 halos, from a per-instance seed."""
    rng = np.random.default_rng(base_seed + index)
    sides = (64, 128, 256, 512, 1024)
    nx = int(rng.choice(sides))
    nv = int(rng.choice(sides))
    s = 4 if max(nx, nv) <= 128 else 8
    if rng.uniform() < 0.5:
        sig = float(rng.uniform(0.3, 0.7))
        return RunConfig(f"batch{index}-spitzer", nx, nv, -1.0, 1.0, -5 * sig, 5 * sig, s, 0.005, 20, 1.0,
                         500, "spitzer", {"sigma": sig}, seed=base_seed + index)
    nh = int(rng.integers(4, 17))
    return RunConfig(f"batch{index}-halos", nx, nv, -1.0, 1.0, -1.5, 1.5, s, 0.002, 20, 1.0, 500,
                     "halos", {"n": nh}, seed=base_seed + index)
