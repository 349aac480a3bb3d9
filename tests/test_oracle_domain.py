"""Pins of the oracle's adaptive computing domain (Sec. 2.2.1, eq. constrf:
f_ini restricted to the rectangle holding every |f| > f_th; Sec. 2.3:
elements on the lattice covering it plus an extra layer, and each map's
sites inside the rectangle spanned by the elements' positions).

Pinned by: (1) an initial condition above the threshold everywhere gives
the fixed-box run bit for bit; (2) the apodised sheet, whose support is
known in closed form, gives the node rectangle of that support, a lattice
range whose lines bracket it with one layer to spare, and a site rectangle
spanned by those lattice positions; (3) under free streaming the site
rectangle follows the elements' exact positions x = q_x + q_v t; (4) the
restricted run stays within the reconstruction tolerance of the fixed-box
run while reconstructing a fraction of the sites.
"""
import math

import numpy as np
import pytest

import oracle.oracle as O
from paper_1705_03750_gb300 import inputs as I

# the apodised thermal-equilibrium sheet on a box about twice its support
WIDE = I.APOD_128.with_(name="apod-wide", nx=192, nv=192, x_lo=-1.2, x_hi=1.2, v_lo=-1.6, v_hi=1.6)
RHO, SIG, ETA = 4.0, 0.2, 0.02


def _oracle(rc, f_th=0.0):
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_fth(f_th)
    o.set_f(I.initial_f(rc))
    return o


def test_threshold_below_every_value_is_the_fixed_box():
    """A wide Gaussian blob is above f_th at every node: the domain is the
    whole box, every element exists, and 30 steps through a remap are the
    fixed-box run bit for bit."""
    rc = I.SPITZER_128.with_(ic="blob", ic_params={"sx": 3.0, "sv": 5.0}, n_s=20)
    a, b = _oracle(rc, 0.0), _oracle(rc, 1e-3)
    assert b.domain()["lattice"] == (0, b.Lx - 1, 0, b.Lv - 1)
    a.step(30)
    b.step(30)
    assert np.array_equal(a.elements(), b.elements())
    assert np.array_equal(a.last_f(), b.last_f())
    assert np.array_equal(a.fini(), b.fini())
    assert b.domain()["rect"] == (0, rc.nx - 1, 0, rc.nv - 1)


def _support():
    """Half-widths of the apodised sheet's support: f_S = eta (1 - atanh(1/2))."""
    f0 = ETA * (1 - math.atanh(0.5))
    k = math.sqrt(math.sqrt(2 * math.pi) * RHO / SIG)
    return math.acosh(math.sqrt(RHO / f0)) / k, SIG * math.sqrt(2 * math.log(RHO / f0))


def test_lagrangian_domain_of_the_apodised_sheet():
    o = _oracle(WIDE, 1e-12)
    fi = o.fini()
    xs, vs = _support()
    x, v = WIDE.x(), WIDE.v()
    # the node rectangle of the closed-form support
    i_in = np.nonzero(np.abs(x) < xs)[0]
    j_in = np.nonzero(np.abs(v) < vs)[0]
    nz = np.nonzero(fi)
    assert (nz[0].min(), nz[0].max(), nz[1].min(), nz[1].max()) == (i_in[0], i_in[-1], j_in[0], j_in[-1])
    # the lattice range: lines k_lo + 1 and k_hi - 1 bracket the rectangle
    # (none closer inside it), with one more line on each side
    klo, khi, llo, lhi = o.domain()["lattice"]
    dxm, dvm = WIDE.s * WIDE.dx, WIDE.s * WIDE.dv
    Kx, Kv = (o.Lx - 3) // 2, (o.Lv - 3) // 2
    qx = lambda k: 0.5 * (WIDE.x_lo + WIDE.x_hi) + (k - Kx - 1) * dxm  # noqa: E731
    qv = lambda l: 0.5 * (WIDE.v_lo + WIDE.v_hi) + (l - Kv - 1) * dvm  # noqa: E731
    eps = 1e-12
    assert qx(klo + 1) <= x[i_in[0]] + eps < qx(klo + 2)
    assert qx(khi - 2) < x[i_in[-1]] - eps <= qx(khi - 1)
    assert qv(llo + 1) <= v[j_in[0]] + eps < qv(llo + 2)
    assert qv(lhi - 2) < v[j_in[-1]] - eps <= qv(lhi - 1)
    # a fraction of the lattice exists
    assert (khi - klo + 1) * (lhi - llo + 1) < 0.35 * o.Lx * o.Lv


def test_first_map_covers_the_lattice_positions():
    """At the first map the elements sit at their lattice positions (moved
    by half a drift): the site rectangle is spanned by the outermost lattice
    lines of the existing range, and holds the whole support."""
    rc = WIDE.with_(G=0.0)
    o = _oracle(rc, 1e-12)
    o.step(1)
    klo, khi, llo, lhi = o.domain()["lattice"]
    i0, i1, j0, j1 = o.domain()["rect"]
    el = o.elements().reshape(o.Lx, o.Lv, 12)[klo:khi + 1, llo:lhi + 1]
    # positions at the map: half a drift before the end of the step
    xm = el[..., 0] - 0.5 * rc.dt * el[..., 1]
    vm = el[..., 1]
    assert i0 == math.ceil((xm.min() - rc.x_lo) / rc.dx - 1e-9)
    assert i1 == math.floor((xm.max() - rc.x_lo) / rc.dx + 1e-9)
    assert j0 == math.ceil((vm.min() - rc.v_lo) / rc.dv - 1e-9)
    assert j1 == math.floor((vm.max() - rc.v_lo) / rc.dv + 1e-9)
    nz = np.nonzero(o.fini())
    assert i0 <= nz[0].min() and nz[0].max() <= i1 and j0 <= nz[1].min() and nz[1].max() <= j1
    f = o.last_f()
    inside = np.zeros_like(f, dtype=bool)
    inside[i0:i1 + 1, j0:j1 + 1] = True
    assert not f[~inside].any()


def test_free_streaming_rectangle_follows_the_exact_positions():
    """G = 0: every element moves as x = q_x + q_v t exactly (drift only), so
    the rectangle after n steps is spanned by the lattice positions of the
    corner elements sheared by t = (n - 1/2) dt at the last map."""
    rc = WIDE.with_(G=0.0, n_s=1000, dt=0.01)
    o = _oracle(rc, 1e-12)
    klo, khi, llo, lhi = o.domain()["lattice"]
    dxm, dvm = rc.s * rc.dx, rc.s * rc.dv
    Kx, Kv = (o.Lx - 3) // 2, (o.Lv - 3) // 2
    qx = 0.5 * (rc.x_lo + rc.x_hi) + (np.arange(klo, khi + 1) - Kx - 1) * dxm
    qv = 0.5 * (rc.v_lo + rc.v_hi) + (np.arange(llo, lhi + 1) - Kv - 1) * dvm
    for n in (5, 17):
        o2 = _oracle(rc, 1e-12)
        o2.step(n)
        t = (n - 0.5) * rc.dt
        xmin = min(qx.min() + qv.min() * t, qx.min() + qv.max() * t)
        xmax = max(qx.max() + qv.min() * t, qx.max() + qv.max() * t)
        i0, i1, j0, j1 = o2.domain()["rect"]
        assert i0 == max(0, math.ceil((xmin - rc.x_lo) / rc.dx - 1e-9))
        assert i1 == min(rc.nx - 1, math.floor((xmax - rc.x_lo) / rc.dx + 1e-9))
        assert (j0, j1) == (max(0, math.ceil((qv.min() - rc.v_lo) / rc.dv - 1e-9)),
                            min(rc.nv - 1, math.floor((qv.max() - rc.v_lo) / rc.dv + 1e-9)))


def test_restricted_run_tracks_the_fixed_box_run():
    """30 steps (a remap at 25) of the apodised sheet: the restricted run's f
    is the fixed-box run's to the reconstruction tolerance, zero outside
    its rectangle, with the same mass, while its maps hold about a fifth of
    the sites."""
    a, b = _oracle(WIDE, 0.0), _oracle(WIDE, 1e-10)
    a.step(30)
    b.step(30)
    fa, fb = a.last_f(), b.last_f()
    assert np.abs(fa - fb).max() <= 1e-6 * np.abs(fa).max()
    i0, i1, j0, j1 = b.domain()["rect"]
    assert (i1 - i0 + 1) * (j1 - j0 + 1) < 0.35 * WIDE.nx * WIDE.nv
    assert b.diagnostics()["mass"] == pytest.approx(a.diagnostics()["mass"], rel=1e-9)
    m, _ = b.compute_map()
    assert (m >= 0).sum() == (i1 - i0 + 1) * (j1 - j0 + 1)   # every site of the rectangle, none outside


def test_nothing_above_the_threshold():
    rc = WIDE
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_fth(10.0)    # above the sheet's maximum (4)
    o.set_f(I.initial_f(rc))
    assert not o.fini().any()
    o.step(3)
    assert not o.last_f().any() and o.domain()["lattice"][1] < o.domain()["lattice"][0]
