"""The paper's apodised thermal-equilibrium sheet (Sec. 3.2, eqs. apofs and
apod), read with the cut of eq. monfg2: pinned against the paper's printed
maximum projected density, the closed-form support and continuity of the
cut, and, through the oracle, the self-consistent force of the sheet in the
paper's units (phi'' = 2 rho) and its near-stationarity."""
import json
import math
import os

import numpy as np
import pytest

import oracle.oracle as O
from paper_1705_03750_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
RHO, SIG, ETA = 4.0, 0.2, 0.02
K = math.sqrt(math.sqrt(2 * math.pi) * RHO / SIG)


def test_projected_density_is_the_printed_maximum():
    """rho(0) = int f(0, v) dv of the apodised sheet rounds to the paper's
    rho_max ~ 2: the apodisation removes only the wings (a leading eta in
    the apodising function, as printed, would give about 3 eta * 2)."""
    v = np.linspace(-1.0, 1.0, 20001)
    rho0 = I.apodised_spitzer(0.0, v).sum() * (v[1] - v[0])
    assert round(rho0, GOLD["thermal_rho_max"]["digits"]) == GOLD["thermal_rho_max"]["value"]
    full = RHO * math.sqrt(2 * math.pi) * SIG
    assert 0.995 * full < rho0 < full


def test_cut_is_continuous_and_has_the_closed_form_support():
    """f = f_S for f_S >= eta; below, f_S (1 + 2 th((f_S - eta)/eta)), which
    is continuous at f_S = eta and reaches 0 at f_S = eta (1 - atanh(1/2))."""
    # along v at x = 0: f_S = RHO exp(-v^2 / 2 sigma^2)
    v_eta = SIG * math.sqrt(2 * math.log(RHO / ETA))
    assert I.apodised_spitzer(0.0, v_eta * (1 - 1e-12)) == pytest.approx(ETA, rel=1e-9)
    assert I.apodised_spitzer(0.0, v_eta * (1 + 1e-12)) == pytest.approx(ETA, rel=1e-9)
    f_zero = ETA * (1 - math.atanh(0.5))
    v_zero = SIG * math.sqrt(2 * math.log(RHO / f_zero))
    assert I.apodised_spitzer(0.0, v_zero * (1 + 1e-9)) == 0.0
    assert I.apodised_spitzer(0.0, v_zero * (1 - 1e-4)) > 0.0
    # along x at v = 0: f_S = RHO / ch^2(K x)
    x_zero = math.acosh(math.sqrt(RHO / f_zero)) / K
    assert I.apodised_spitzer(x_zero * (1 + 1e-9), 0.0) == 0.0
    assert I.apodised_spitzer(x_zero * (1 - 1e-4), 0.0) > 0.0
    # the workload's box holds the whole support
    rc = I.APOD_128
    assert rc.x_hi > x_zero and rc.v_hi > v_zero


def test_force_of_the_sheet_in_paper_units():
    """With G = 1/(2 pi) (phi'' = 2 rho) the oracle's force on the sheet is
    a(x) = -2 int_0^x rho = -(2 rho0 / K) th(K x) up to the apodisation and
    the grid: the reading of the units the workload relies on."""
    rc = I.APOD_128.with_(nx=257, nv=257)
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_f(I.initial_f(rc))
    o.reconstruct()
    a = o.density_force()["a"]
    rho0 = RHO * math.sqrt(2 * math.pi) * SIG
    x = rc.x()
    exact = -(2 * rho0 / K) * np.tanh(K * x)
    inner = np.abs(x) < 0.3
    assert np.abs(a[inner] - exact[inner]).max() < 1e-2 * np.abs(exact).max()
    # and G = 1 (the other reading of "within some trivial factor") is 2 pi off
    assert np.abs(2 * math.pi * a[inner] - exact[inner]).max() > 0.5 * np.abs(exact).max()


def test_sheet_stays_nearly_stationary_in_the_oracle():
    """The apodised sheet is close to equilibrium: after 50 steps (two remaps
    at n_s = 25) f moves by a small fraction of its maximum, and the mass is
    kept to the interpolation accuracy."""
    rc = I.APOD_128
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    f0 = I.initial_f(rc)
    o.set_f(f0)
    o.step(50)
    f = o.last_f()
    assert np.abs(f - f0).max() < 2e-2 * f0.max()
    m0 = f0.sum() * rc.dx * rc.dv
    assert abs(o.diagnostics()["mass"] - m0) < 1e-3 * m0
    np.testing.assert_allclose(f, f[::-1, ::-1], atol=1e-9 * f0.max())
