"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes one piece of the oracle to something other than itself, so
that a plausible slip (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.  No GPU is needed.
"""
import math

import numpy as np
import pytest

import oracle.oracle as O
from paper_1705_03750_gb300 import inputs as I

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------
# Sec. 2.2.1: six-point quadratic interpolation
# ---------------------------------------------------------------------------

def _six_point_bruteforce(F, u, w):
    """Fit a + b x + c y + d x^2 + e y^2 + g x y through the six nodes chosen
    as the paper describes (nearest node, its cross, and the fourth corner of
    the unit square that contains the point), by a dense linear solve."""
    inn, jn = math.floor(u + 0.5), math.floor(w + 0.5)
    ic, jc = math.floor(u), math.floor(w)
    cross = [(inn, jn), (inn + 1, jn), (inn - 1, jn), (inn, jn + 1), (inn, jn - 1)]
    square = [(ic, jc), (ic + 1, jc), (ic, jc + 1), (ic + 1, jc + 1)]
    corner = [p for p in square if p not in cross]
    assert len(corner) == 1
    pts = cross + corner
    A = np.array([[1, x - inn, y - jn, (x - inn) ** 2, (y - jn) ** 2, (x - inn) * (y - jn)] for x, y in pts], float)
    b = np.array([F[x, y] for x, y in pts])
    coef = np.linalg.solve(A, b)
    dx, dy = u - inn, w - jn
    return coef @ np.array([1, dx, dy, dx * dx, dy * dy, dx * dy])


def test_qinterp_matches_six_point_fit_all_quadrants():
    F = RNG.normal(size=(12, 11))
    for _ in range(400):
        u = RNG.uniform(2.0, 9.0)
        w = RNG.uniform(2.0, 8.0)
        assert O.qinterp(F, u, w) == pytest.approx(_six_point_bruteforce(F, u, w), abs=1e-12)


def test_qinterp_reproduces_bivariate_quadratics():
    c = RNG.normal(size=6)
    ii, jj = np.meshgrid(np.arange(10.0), np.arange(9.0), indexing="ij")
    p = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y
    F = p(ii, jj)
    for _ in range(300):
        u, w = RNG.uniform(1.0, 8.0), RNG.uniform(1.0, 7.0)
        assert O.qinterp(F, u, w) == pytest.approx(p(u, w), rel=1e-11, abs=1e-10)


def test_qinterp_nodes_and_outside():
    F = RNG.normal(size=(6, 7))
    for i in range(6):
        for j in range(7):
            assert O.qinterp(F, i, j) == F[i, j]
    assert O.qinterp(F, -2.5, 3.0) == 0.0
    assert O.qinterp(F, 3.0, 7.6) == 0.0
    # half a cell beyond the last node only the in-grid nodes contribute
    G = np.ones((6, 7))
    assert O.qinterp(G, 5.0, 3.0) == pytest.approx(1.0)
    # nearest node 5, dq = 0.4: F(5)(1 - dq^2) + F(4) dq(dq - 1)/2 with F(6) = 0
    assert O.qinterp(G, 5.4, 3.0) == pytest.approx(0.84 - 0.12)


# ---------------------------------------------------------------------------
# Sec. 2.2.2: cubic B-splines with zero slope at the end nodes
# ---------------------------------------------------------------------------

def _dense_spline_matrix(n):
    B = lambda t: O.bspline3(t)
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(i - 2, i + 3):
            g = 1 if k == -1 else (n - 2 if k == n else k)
            if 0 <= g < n and -1 <= k <= n:
                A[i, g] += B(i - k)
    return A


def test_bspline3_textbook():
    # (1/6) sum_{r=0}^{4} (-1)^r C(4,r) (t + 2 - r)_+^3, the centred cubic B-spline
    for t in np.linspace(-2.5, 2.5, 101):
        ref = sum((-1) ** r * math.comb(4, r) * max(t + 2 - r, 0.0) ** 3 for r in range(5)) / 6.0
        assert O.bspline3(t) == pytest.approx(ref, abs=1e-14)


@pytest.mark.parametrize("n", [4, 5, 17, 64])
def test_spline_solve_1d_matches_dense(n):
    f = RNG.normal(size=n)
    eta = O.spline_solve_1d(f)
    ref = np.linalg.solve(_dense_spline_matrix(n), f)
    np.testing.assert_allclose(eta, ref, rtol=1e-12, atol=1e-12)


def test_spline_bump_is_unit_coefficient_and_is_reproduced():
    nx, nv, k0, l0 = 20, 24, 7, 13
    ii, jj = np.meshgrid(np.arange(nx), np.arange(nv), indexing="ij")
    bump = np.vectorize(O.bspline3)
    f = bump(ii - k0) * bump(jj - l0)
    eta = O.spline_solve_2d(f)
    e = np.zeros_like(f)
    e[k0, l0] = 1.0
    np.testing.assert_allclose(eta, e, atol=1e-13)
    for _ in range(200):
        u, w = RNG.uniform(0, nx - 1), RNG.uniform(0, nv - 1)
        assert O.spline_eval(eta, u, w) == pytest.approx(O.bspline3(u - k0) * O.bspline3(w - l0), abs=1e-13)


def test_spline_eval_at_nodes_returns_f_and_end_slope_is_zero():
    f = RNG.normal(size=(9, 11))
    eta = O.spline_solve_2d(f)
    for i in range(9):
        for j in range(11):
            assert O.spline_eval(eta, i, j) == pytest.approx(f[i, j], abs=1e-12)
    h = 1e-6
    for j in (0.3, 4.7):
        slope = (O.spline_eval(eta, h, j) - O.spline_eval(eta, 0.0, j)) / h
        assert abs(slope) < 1e-4
        slope = (O.spline_eval(eta, 8.0, j) - O.spline_eval(eta, 8.0 - h, j)) / h
        assert abs(slope) < 1e-4
    # the finite B-spline sum is continuous across the edge nodes and vanishes
    # three cells beyond them
    assert O.spline_eval(eta, -1e-12, 3.0) == pytest.approx(f[0, 3], abs=1e-9)
    assert O.spline_eval(eta, 3.0, 10.0 + 1e-12) == pytest.approx(f[3, 10], abs=1e-9)
    assert O.spline_eval(eta, -3.0, 3.0) == 0.0 and O.spline_eval(eta, 2.0, 13.0) == 0.0 and O.spline_eval(eta, 2.0, 12.5) != 0.0


# ---------------------------------------------------------------------------
# Sec. 2.1: second-order inverse map
# ---------------------------------------------------------------------------

def _random_element(scaleH=1.0):
    T = np.eye(2) + 0.6 * RNG.normal(size=(2, 2))
    while abs(np.linalg.det(T)) < 0.3:
        T = np.eye(2) + 0.6 * RNG.normal(size=(2, 2))
    Hx = scaleH * RNG.normal(size=3)
    Hv = scaleH * RNG.normal(size=3)
    P = RNG.normal(size=2)
    el = np.array([P[0], P[1], T[0, 0], T[0, 1], T[1, 0], T[1, 1], *Hx, *Hv])
    return el, T, Hx, Hv, P


def _forward(T, Hx, Hv, P, dQ):
    Hxm = np.array([[Hx[0], Hx[1]], [Hx[1], Hx[2]]])
    Hvm = np.array([[Hv[0], Hv[1]], [Hv[1], Hv[2]]])
    return P + T @ dQ + 0.5 * np.array([dQ @ Hxm @ dQ, dQ @ Hvm @ dQ])


def test_inverse_map_exact_for_linear_flow():
    for _ in range(50):
        el, T, Hx, Hv, P = _random_element(scaleH=0.0)
        Q = RNG.normal(size=2)
        tay = O.taylor_one(el, *Q)
        dQ = RNG.normal(size=2)
        Pt = P + T @ dQ
        dq = O.qofp(tay, *Pt)
        np.testing.assert_allclose(dq, dQ, atol=1e-12)


def test_inverse_map_error_is_third_order():
    ratios = []
    for _ in range(30):
        el, T, Hx, Hv, P = _random_element()
        tay = O.taylor_one(el, 0.0, 0.0)
        d = RNG.normal(size=2)
        d /= np.linalg.norm(d)
        errs = []
        for eps in (1e-2, 5e-3):
            dQ = eps * d
            Pt = _forward(T, Hx, Hv, P, dQ)
            errs.append(np.linalg.norm(np.array(O.qofp(tay, *Pt)) - dQ))
        ratios.append(errs[0] / errs[1])
    # halving the offset divides the error by 2^3 (a first-order inverse, or a
    # wrong sign or transposition in the second-order term, gives 2^2)
    assert 7.0 < np.median(ratios) < 9.0


def test_taylor_terms_match_matrix_algebra():
    el, T, Hx, Hv, P = _random_element()
    tay = O.taylor_one(el, 0.25, -0.5)
    Ti = np.linalg.inv(T)
    np.testing.assert_allclose(tay[2:6], Ti.ravel(), rtol=1e-13, atol=1e-13)
    for l, H in enumerate((Hx, Hv)):
        Hm = np.array([[H[0], H[1]], [H[1], H[2]]])
        G = Ti.T @ Hm @ Ti
        np.testing.assert_allclose(tay[6 + 3 * l:9 + 3 * l], [G[0, 0], G[0, 1], G[1, 1]], rtol=1e-12, atol=1e-12)
    assert tay[12] == 0.25 and tay[13] == -0.5


# ---------------------------------------------------------------------------
# Sec. 2.3.2 / 2.3.3: Monaghan kernel and the alpha / beta ranges
# ---------------------------------------------------------------------------

def test_W_is_the_M4_spline():
    for x in np.linspace(0, 2.5, 251):
        ref = 0.25 * (max(2 - x, 0) ** 3 - 4 * max(1 - x, 0) ** 3)
        assert O.W(x) == pytest.approx(ref, abs=1e-15)


def test_paper_constants_golden():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    assert round(O.ALPHA, g["alpha"]["digits"]) == g["alpha"]["value"]
    assert round(O.BETA, g["beta"]["digits"]) == g["beta"]["value"]
    assert round(1 - math.sqrt(3) / 2, g["beta_bound"]["digits"]) == g["beta_bound"]["value"]
    # alpha = 1/2 - E_max with E_max = beta
    assert O.ALPHA == pytest.approx(0.5 - O.BETA, abs=1e-15)
    assert O.BETA <= 1 - math.sqrt(3) / 2
    assert I.ALPHA == O.ALPHA and I.BETA == O.BETA


def test_beta_set_drops_only_zero_weight_elements():
    """With exact proposals, every lattice neighbour left out of the beta set
    lies at d >= 1 element spacing, so its Monaghan weight W(2d) is zero."""
    for _ in range(20000):
        xi, ze = RNG.uniform(-0.5, 0.5, size=2)
        kept = set(O.beta_offsets(xi, ze))
        assert (0, 0) in kept and len(kept) in (4, 5)
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                if (a, b) not in kept:
                    d = math.hypot(xi - a, ze - b)
                    assert O.W(2 * d) == 0.0, (xi, ze, a, b)


def test_beta_bound_is_sharp():
    """A margin beyond 1 - sqrt(3)/2 drops an element with non-zero weight."""
    bad = 0
    for _ in range(20000):
        xi, ze = RNG.uniform(-0.5, 0.5, size=2)
        kept = set(O.beta_offsets(xi, ze, beta=0.2))
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                if (a, b) not in kept and O.W(2 * math.hypot(xi - a, ze - b)) > 0:
                    bad += 1
    assert bad > 0


def test_alpha_test_never_misses_a_closer_neighbour_for_exact_maps():
    """For exact proposals a site passes the alpha-restricted test only if no
    element of the full 3x3 neighbourhood is closer."""
    for _ in range(20000):
        xi, ze = RNG.uniform(-1.0, 1.0, size=2)
        d2 = xi * xi + ze * ze
        tested = O.alpha_offsets(xi, ze)
        passes = all((xi - a) ** 2 + (ze - b) ** 2 >= d2 for a, b in tested)
        if passes:
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    assert (xi - a) ** 2 + (ze - b) ** 2 >= d2 - 1e-12


# ---------------------------------------------------------------------------
# Sec. 2.5: force from the masses, derivatives, TSC
# ---------------------------------------------------------------------------

def test_force_matches_bruteforce_mass_difference():
    M = RNG.uniform(0, 1, size=37)
    G = 0.7
    a, da, d2a = O.force_from_mass(M, 0.1, G)
    for i in range(M.size):
        ref = 2 * math.pi * G * (M[i + 1:].sum() - M[:i].sum())
        assert a[i] == pytest.approx(ref, abs=1e-13)
    aext = np.concatenate([[2 * math.pi * G * M.sum()], a, [-2 * math.pi * G * M.sum()]])
    np.testing.assert_allclose(da, (aext[2:] - aext[:-2]) / 0.2, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(d2a, (aext[2:] + aext[:-2] - 2 * aext[1:-1]) / 0.01, rtol=1e-12, atol=1e-10)


def _spitzer_force_errors(n):
    sigma, G = 0.5, 1.0
    x0 = sigma ** 2 / math.pi
    x = np.linspace(-1.5, 1.5, n)
    dx = x[1] - x[0]
    rho = (0.5 / x0) / np.cosh(x / x0) ** 2
    a, da, d2a = O.force_from_mass(rho * dx, dx, G)
    exact_a = -2 * math.pi * G * np.tanh(x / x0)           # M_total = 1
    exact_da = -4 * math.pi * G * rho                       # Poisson: a' = -4 pi G rho
    exact_d2a = -4 * math.pi * G * rho * (-2 * np.tanh(x / x0) / x0)
    core = np.abs(x) < 1.0
    return (np.abs(a - exact_a)[core].max(), np.abs(da - exact_da)[core].max(),
            np.abs(d2a - exact_d2a)[core].max())


def test_force_of_spitzer_sheet_converges_at_second_order():
    e1 = _spitzer_force_errors(601)
    e2 = _spitzer_force_errors(1201)
    for k in range(3):
        assert 3.0 < e1[k] / e2[k] < 5.0, (k, e1, e2)
    assert e2[1] < 1e-2 * 4 * math.pi * 6.3


def test_spitzer_ic_is_stationary_with_the_mass_force():
    """The isothermal sheet is stationary iff a = -2 sigma^2 tanh(x/x0)/x0;
    the mass-difference force with factor 2 pi G gives exactly that."""
    c = I.SPITZER_128.with_(nx=2001, x_lo=-1.5, x_hi=1.5)
    x = c.x()
    f = I.spitzer(x[:, None], np.linspace(-3, 3, 601)[None, :], sigma=0.5, G=1.0)
    M = f.sum(axis=1) * (6.0 / 600) * c.dx
    a, _, _ = O.force_from_mass(M, c.dx, 1.0)
    x0 = 0.25 / math.pi
    ref = -2 * 0.25 * np.tanh(x / x0) / x0
    assert np.abs(a - ref)[np.abs(x) < 1].max() < 2e-3 * np.abs(ref).max()


def test_paper_thermal_equilibrium_rho_max_golden():
    """The paper's f_S with rho_S = 4, sigma_S = 0.2 (paper units, 2 pi G = 1)
    has maximum projected density ~2 as printed, and equals our Spitzer
    generator with G = 1/(2 pi) and the same total mass."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    rho_S, sig = 4.0, 0.2
    k = math.sqrt(math.sqrt(2 * math.pi) * rho_S / sig)
    fS = lambda x, v: rho_S / np.cosh(k * x) ** 2 * np.exp(-0.5 * (v / sig) ** 2)
    rho_max = rho_S * math.sqrt(2 * math.pi) * sig
    assert round(rho_max, g["thermal_rho_max"]["digits"]) == g["thermal_rho_max"]["value"]
    M = 2 * rho_max / k
    x = np.linspace(-0.5, 0.5, 41)[:, None]
    v = np.linspace(-0.8, 0.8, 33)[None, :]
    np.testing.assert_allclose(I.spitzer(x, v, sigma=sig, G=1 / (2 * math.pi), mass=M), fS(x, v), rtol=1e-12)


def test_tsc_linear_exact_and_extensions():
    A = 0.3 + 1.7 * np.arange(20.0)
    for u in RNG.uniform(1.0, 18.0, size=100):
        assert O.tsc(A, 9.0, -9.0, u) == pytest.approx(0.3 + 1.7 * u, abs=1e-12)
    for u in RNG.uniform(-5, 25, size=100):
        wts = [O.tsc(np.eye(20)[k], 0, 0, u) for k in range(20)]
        if 1.0 <= u <= 18.0:
            assert sum(wts) == pytest.approx(1.0, abs=1e-14)
    assert O.tsc(A, 9.0, -9.0, -3.0) == 9.0
    assert O.tsc(A, 9.0, -9.0, 40.0) == -9.0


# ---------------------------------------------------------------------------
# Sec. 2.4: elements of metric under a frozen force
# ---------------------------------------------------------------------------

def _oracle(nx=65, nv=65, box=(-2.0, 2.0, -2.0, 2.0), s=4, dt=0.01, n_s=1000, G=0.0, **kw):
    return O.Oracle(nx, nv, box[0], box[1], box[2], box[3], s, dt, n_s, G, **kw)


def test_free_streaming_elements_are_exact():
    o = _oracle(G=0.0, dt=0.01)
    o.set_f(np.zeros((65, 65)))
    e0 = o.elements()
    o.step(37)
    e = o.elements()
    t = 0.37
    np.testing.assert_allclose(e[:, 0], e0[:, 0] + e0[:, 1] * t, atol=1e-13)
    np.testing.assert_allclose(e[:, 1], e0[:, 1], atol=0)
    np.testing.assert_allclose(e[:, 3], t, atol=1e-14)
    np.testing.assert_array_equal(e[:, [2, 5]], 1.0)
    np.testing.assert_array_equal(e[:, 4], 0.0)
    np.testing.assert_array_equal(e[:, 6:], 0.0)


def test_harmonic_dkd_matches_closed_form_matrix():
    o = _oracle(nx=401, box=(-4.0, 4.0, -2.0, 2.0), dt=0.05)
    o.set_f(np.zeros((401, 65)))
    w2 = 2.3
    x = np.linspace(-4, 4, 401)
    a = -w2 * x
    dx = x[1] - x[0]
    o.push_frozen(a, np.full_like(x, -w2), np.zeros_like(x), -w2 * (x[0] - dx), -w2 * (x[-1] + dx), 30)
    h, dt = 0.025, 0.05
    D = np.array([[1, h], [0, 1]])
    K = np.array([[1, 0], [-w2 * dt, 1]])
    Mn = np.linalg.matrix_power(D @ K @ D, 30)
    o0 = _oracle(nx=401, box=(-4.0, 4.0, -2.0, 2.0))
    o0.set_f(np.zeros((401, 65)))
    e0 = o0.elements()
    e = o.elements()
    inside = (np.abs(e0[:, 0]) < 1.2) & (np.abs(e0[:, 1]) < 1.2)
    assert inside.sum() > 20
    P = (Mn @ e0[inside][:, :2].T).T
    np.testing.assert_allclose(e[inside][:, :2], P, atol=1e-12)
    np.testing.assert_allclose(e[inside][:, 2:6], np.broadcast_to(Mn.ravel(), (inside.sum(), 4)), atol=1e-12)
    np.testing.assert_array_equal(e[inside][:, 6:], 0.0)
    det = e[:, 2] * e[:, 5] - e[:, 3] * e[:, 4]
    np.testing.assert_allclose(det, 1.0, atol=1e-13)


def test_deformation_and_hessian_match_finite_differences_of_trajectories():
    """T and H of an element agree with finite differences of the positions
    of nearby elements pushed by the same anharmonic frozen force."""
    n = 8001
    x = np.linspace(-4, 4, n)
    k = 1.3
    a, da, d2a = -np.sin(k * x), -k * np.cos(k * x), k * k * np.sin(k * x)
    o = _oracle(nx=n, box=(-4.0, 4.0, -2.0, 2.0), dt=0.02)
    o.set_f(np.zeros((n, 65)))
    e = o.elements()
    h = 0.01
    Q0 = np.array([0.4, 0.3])
    offs = [(a_, b_) for a_ in (-1, 0, 1) for b_ in (-1, 0, 1)]
    for q, (i, j) in enumerate(offs):
        e[q] = [Q0[0] + i * h, Q0[1] + j * h, 1, 0, 0, 1, 0, 0, 0, 0, 0, 0]
    o.set_elements(e)
    o.push_frozen(a, da, d2a, 0.0, 0.0, 60)
    e = o.elements()
    P = {off: e[q, :2] for q, off in enumerate(offs)}
    T_fd = np.column_stack([(P[(1, 0)] - P[(-1, 0)]) / (2 * h), (P[(0, 1)] - P[(0, -1)]) / (2 * h)])
    H_xx = (P[(1, 0)] - 2 * P[(0, 0)] + P[(-1, 0)]) / h ** 2
    H_vv = (P[(0, 1)] - 2 * P[(0, 0)] + P[(0, -1)]) / h ** 2
    H_xv = (P[(1, 1)] - P[(1, -1)] - P[(-1, 1)] + P[(-1, -1)]) / (4 * h * h)
    c = e[offs.index((0, 0))]
    np.testing.assert_allclose(c[2:6], T_fd.ravel(), rtol=2e-4, atol=2e-4)
    Hx = np.array([H_xx[0], H_xv[0], H_vv[0]])
    Hv = np.array([H_xx[1], H_xv[1], H_vv[1]])
    scale = np.abs(np.concatenate([Hx, Hv])).max()
    assert scale > 0.1
    np.testing.assert_allclose(c[6:9], Hx, atol=3e-3 * scale)
    np.testing.assert_allclose(c[9:12], Hv, atol=3e-3 * scale)


# ---------------------------------------------------------------------------
# Sec. 2.3.1: the influence map
# ---------------------------------------------------------------------------

def test_map_at_initialisation_is_nearest_lattice_element():
    c = I.SPITZER_128
    o = O.Oracle(c.nx, c.nv, c.x_lo, c.x_hi, c.v_lo, c.v_hi, c.s, c.dt, c.n_s, c.G)
    o.set_f(I.initial_f(c))
    m, st = o.compute_map()
    assert st == 0
    Kx = (o.Lx - 3) // 2
    k = np.floor((np.arange(128) - 63.5) / 4 + 0.5).astype(int) + Kx + 1
    expect = k[:, None] * o.Lv + k[None, :]
    np.testing.assert_array_equal(m, expect)
    assert o.map_stats()["holes"] == 0 and o.map_stats()["multi_claims"] == 0


def test_map_exact_ties_go_to_the_smaller_index():
    # dx = dv = 1 and s = 4 make every distance exact: sites midway between two
    # lattice elements are true ties, claimed by both, kept by the smaller m
    o = O.Oracle(33, 33, -16.0, 16.0, -16.0, 16.0, 4, 0.01, 10, 0.0)
    o.set_f(np.zeros((33, 33)))
    m, st = o.compute_map()
    Kx = (o.Lx - 3) // 2
    r = (np.arange(33) - 16) / 4.0
    k = np.ceil(r - 0.5).astype(int) + Kx + 1      # nearest, ties to the lower
    np.testing.assert_array_equal(m, k[:, None] * o.Lv + k[None, :])
    assert o.map_stats()["multi_claims"] > 0


def test_map_of_sheared_lattice_is_nearest_in_lagrangian_space():
    c = I.FREE_128
    o = O.Oracle(c.nx, c.nv, c.x_lo, c.x_hi, c.v_lo, c.v_hi, c.s, c.dt, c.n_s, 0.0)
    o.set_f(I.initial_f(c))
    o.step(4)                      # free streaming, t = 0.02
    m, st = o.compute_map()
    t = 0.02
    X, V = np.meshgrid(c.x(), c.v(), indexing="ij")
    qx, qv = X - V * t, V
    Kx = (o.Lx - 3) // 2
    kx = np.floor((qx - 0.0) / (c.s * c.dx) + 0.5).astype(int) + Kx + 1
    kv = np.floor((qv - 0.0) / (c.s * c.dv) + 0.5).astype(int) + Kx + 1
    expect = kx * o.Lv + kv
    assert st == 0
    np.testing.assert_array_equal(m, expect)


def _bruteforce_map(o, pad):
    """Percolation restated with scipy's connected-component labelling: for
    each element the pass set on the padded lattice, its 4-connected
    component through the start site, claims by (d^2, index), then Jacobi
    hole rounds."""
    from scipy import ndimage
    nx, nv = o.nx, o.nv
    cfg = o.cfg
    dx = (cfg.x_hi - cfg.x_lo) / (nx - 1)
    dv = (cfg.v_hi - cfg.v_lo) / (nv - 1)
    inv_dxm, inv_dvm = 1.0 / (float(cfg.s) * dx), 1.0 / (float(cfg.s) * dv)
    tay = o.taylor()
    el = o.elements()
    Lx, Lv = o.Lx, o.Lv

    def d2(m, i, j):
        qx, qv = O.qofp(tay[m], cfg.x_lo + float(i) * dx, cfg.v_lo + float(j) * dv)
        xi, ze = qx * inv_dxm, qv * inv_dvm
        return xi * xi + ze * ze, xi, ze

    def passes(m, i, j):
        dm, xi, ze = d2(m, i, j)
        k, l = divmod(m, Lv)
        for a, b in O.alpha_offsets(xi, ze):
            kk, ll = k + a, l + b
            if 0 <= kk < Lx and 0 <= ll < Lv and d2(kk * Lv + ll, i, j)[0] < dm:
                return False
        return True

    key = lambda d: np.frombuffer(np.float64(d).tobytes(), dtype=np.uint64)[0]
    best = {}
    for m in range(o.ne):
        i0 = math.floor((el[m, 0] - cfg.x_lo) * (1.0 / dx) + 0.5)
        j0 = math.floor((el[m, 1] - cfg.v_lo) * (1.0 / dv) + 0.5)
        if not (-pad <= i0 < nx + pad and -pad <= j0 < nv + pad):
            continue
        # pass set in a box around the start wide enough for these tiny cases
        lo_i, hi_i = max(-pad, i0 - 24), min(nx + pad - 1, i0 + 24)
        lo_j, hi_j = max(-pad, j0 - 24), min(nv + pad - 1, j0 + 24)
        mask = np.zeros((hi_i - lo_i + 1, hi_j - lo_j + 1), bool)
        for i in range(lo_i, hi_i + 1):
            for j in range(lo_j, hi_j + 1):
                mask[i - lo_i, j - lo_j] = passes(m, i, j)
        if not mask[i0 - lo_i, j0 - lo_j]:
            continue
        lab, _ = ndimage.label(mask)
        comp = lab == lab[i0 - lo_i, j0 - lo_j]
        for (ii, jj) in zip(*np.nonzero(comp)):
            i, j = ii + lo_i, jj + lo_j
            if 0 <= i < nx and 0 <= j < nv:
                kd = (key(d2(m, i, j)[0]), m)
                if (i, j) not in best or kd < best[(i, j)]:
                    best[(i, j)] = kd
    mp = -np.ones((nx, nv), np.int32)
    for (i, j), (_, m) in best.items():
        mp[i, j] = m
    while (mp < 0).any():
        prev = mp.copy()
        for i, j in zip(*np.nonzero(prev < 0)):
            cands = []
            for a, b in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                if 0 <= i + a < nx and 0 <= j + b < nv and prev[i + a, j + b] >= 0:
                    cm = int(prev[i + a, j + b])
                    cands.append((key(d2(cm, i, j)[0]), cm))
            if cands:
                mp[i, j] = min(cands)[1]
    return mp


@pytest.mark.parametrize("s,steps", [(4, 40), (4, 60), (2, 50)])
def test_map_matches_bruteforce_percolation_on_evolved_elements(s, steps):
    """Elements of a small Spitzer run carried far past a remap period, so
    that overlapping claims and unexplored sites both occur."""
    c = I.SPITZER_128.with_(nx=32, nv=32, s=s, n_s=1000, dt=0.01)
    o = O.Oracle(c.nx, c.nv, c.x_lo, c.x_hi, c.v_lo, c.v_hi, c.s, c.dt, c.n_s, c.G)
    o.set_f(I.initial_f(c))
    o.step(steps)
    m, st = o.compute_map()
    assert st == 0
    stats = o.map_stats()
    assert stats["multi_claims"] > 0 and stats["holes"] > 0     # both rules exercised
    np.testing.assert_array_equal(m, _bruteforce_map(o, pad=s))


# ---------------------------------------------------------------------------
# Whole method
# ---------------------------------------------------------------------------

def _run(cfg, steps):
    o = O.Oracle(cfg.nx, cfg.nv, cfg.x_lo, cfg.x_hi, cfg.v_lo, cfg.v_hi, cfg.s, cfg.dt, cfg.n_s, cfg.G)
    o.set_f(I.initial_f(cfg))
    o.step(steps)
    return o


def _free_error(n):
    cfg = I.FREE_128.with_(nx=n, nv=n, x_lo=-1.0, x_hi=1.0, v_lo=-1.0, v_hi=1.0, ic="blob",
                           ic_params={"x0": -0.2, "sx": 0.12, "v0": 0.1, "sv": 0.15}, dt=0.01, n_s=10)
    o = _run(cfg, 25)
    t = 24 * cfg.dt + 0.5 * cfg.dt          # the last f is at t_n + dt/2
    X, V = np.meshgrid(cfg.x(), cfg.v(), indexing="ij")
    exact = I.ic_function(cfg)(X - V * t, V)
    return np.abs(o.last_f() - exact).max(), o


def test_free_streaming_matches_exact_solution_and_converges():
    e1, o = _free_error(64)
    e2, _ = _free_error(128)
    assert e1 < 2e-2
    assert e1 / e2 > 3.0          # quadratic/cubic interpolation errors shrink with dx
    m = o.diagnostics()["mass"]
    assert abs(m - 2 * math.pi * 0.12 * 0.15) < 2e-3


def test_spitzer_sheet_stays_stationary_and_symmetric():
    cfg = I.SPITZER_128
    o = _run(cfg, 60)
    f0 = I.initial_f(cfg)
    f = o.last_f()
    assert np.abs(f - f0).max() < 2e-2 * f0.max()
    # the isothermal sheet is symmetric under P -> -P, and so is the method
    np.testing.assert_allclose(f, f[::-1, ::-1], atol=1e-9 * f0.max())
    d = o.diagnostics()
    assert abs(d["detT_min"] - 1) < 1e-12 and abs(d["detT_max"] - 1) < 1e-12
    o2 = _run(cfg, 1)
    E0 = o2.diagnostics()["energy"]
    assert abs(d["energy"] - E0) < 1e-3 * abs(E0)
    assert abs(d["mass"] - 1.0) < 1e-3


def test_remap_right_after_initialisation_is_identity():
    cfg = I.SPITZER_128
    o = O.Oracle(cfg.nx, cfg.nv, cfg.x_lo, cfg.x_hi, cfg.v_lo, cfg.v_hi, cfg.s, cfg.dt, cfg.n_s, cfg.G)
    f0 = I.initial_f(cfg)
    o.set_f(f0)
    fnew, Qr = o.remap_resample()
    X, V = np.meshgrid(cfg.x(), cfg.v(), indexing="ij")
    np.testing.assert_allclose(Qr[..., 0], X, atol=1e-14)
    np.testing.assert_allclose(Qr[..., 1], V, atol=1e-14)
    np.testing.assert_allclose(fnew, f0, atol=1e-12 * f0.max())


def test_frozen_potential_backward_map_is_second_order_in_element_spacing():
    """Q(P) from the elements after pushing them through a frozen harmonic
    potential equals the exact pre-image (the flow is linear, so the Taylor
    map is exact): checks the composition step -> Taylor -> map -> Q."""
    nx = 257
    o = O.Oracle(nx, 65, -2.0, 2.0, -2.0, 2.0, 4, 0.02, 1000, 0.0)
    o.set_f(np.zeros((nx, 65)))
    x = np.linspace(-2, 2, nx)
    w2 = 1.7
    dx = x[1] - x[0]
    o.push_frozen(-w2 * x, np.full(nx, -w2), np.zeros(nx), -w2 * (x[0] - dx), -w2 * (x[-1] + dx), 25)
    tay = o.taylor()
    m, st = o.compute_map()
    D = np.array([[1, 0.01], [0, 1]])
    K = np.array([[1, 0], [-w2 * 0.02, 1]])
    Minv = np.linalg.inv(np.linalg.matrix_power(D @ K @ D, 25))
    X, V = np.meshgrid(x, np.linspace(-2, 2, 65), indexing="ij")
    errs = []
    for i in range(60, 200, 7):
        for j in range(15, 50, 5):
            mm = m[i, j]
            dq = O.qofp(tay[mm], X[i, j], V[i, j])
            Q = np.array([tay[mm, 12] + dq[0], tay[mm, 13] + dq[1]])
            errs.append(np.abs(Q - Minv @ np.array([X[i, j], V[i, j]])).max())
    assert max(errs) < 1e-12


# ---------------------------------------------------------------------------
# Sec. 3.2 Casimirs and Sec. 2.3.2 E_map
# ---------------------------------------------------------------------------

def test_casimirs_of_a_gaussian_match_closed_forms():
    """S = -int f log f, L1 and L2 of a normalised isotropic Gaussian
    (variance s2 per axis) are log(2 pi e s2), 1 and 1/(4 pi s2); the grid
    sums converge to them (midpoint quadrature of a smooth, decayed f)."""
    s2 = 0.09
    n = 401
    o = _oracle(nx=n, nv=n, box=(-3.0, 3.0, -3.0, 3.0))
    x = np.linspace(-3, 3, n)
    X, V = np.meshgrid(x, x, indexing="ij")
    f = np.exp(-(X ** 2 + V ** 2) / (2 * s2)) / (2 * math.pi * s2)
    o.set_f(f)
    d = o.diagnostics()
    assert d["entropy"] == pytest.approx(math.log(2 * math.pi * math.e * s2), rel=1e-6)
    assert d["l1"] == pytest.approx(1.0, rel=1e-9)
    assert d["l2"] == pytest.approx(1.0 / (4 * math.pi * s2), rel=1e-6)
    # |f| and f log|f| for a sign change: S uses |f| inside the log only
    o.set_f(-f)
    d2 = o.diagnostics()
    assert d2["l1"] == pytest.approx(d["l1"]) and d2["l2"] == pytest.approx(d["l2"])
    assert d2["entropy"] == pytest.approx(-d["entropy"])


def test_emap_vanishes_where_the_second_order_maps_are_exact():
    """E_map compares the positions two neighbouring elements propose for the
    same site.  Where every element follows the same flow and its
    second-order map is exact (elements on the lattice at initialisation;
    free streaming, whose maps are linear) all proposals coincide, and E_map
    is rounding only; a wrong sign or index in the mismatch
    ((a + xi_n) - xi_m) would make it of order one.  (A frozen force is no
    such case: the outer elements, beyond the grid, feel its constant
    extension, not the interior's law.)"""
    o = _oracle(nx=129, nv=65, box=(-2.0, 2.0, -2.0, 2.0), s=4, dt=0.02)
    o.set_f(np.zeros((129, 65)))
    assert o.diagnostics()["emap"] == 0.0  # no map yet
    o.compute_map()
    assert o.diagnostics()["emap"] < 1e-12
    fr = _oracle(nx=129, nv=65, box=(-2.0, 2.0, -2.0, 2.0), s=4, dt=0.01, G=0.0)
    fr.set_f(np.zeros((129, 65)))
    fr.step(30)  # free streaming: exact linear maps; the step's map is the transport map
    assert fr.diagnostics()["emap"] < 1e-10


def test_emap_is_positive_for_a_nonlinear_flow():
    """An anharmonic frozen force makes the maps curved: neighbouring
    elements then disagree at third order and E_map is clearly non-zero."""
    n = 129
    o = _oracle(nx=n, nv=65, box=(-2.0, 2.0, -2.0, 2.0), s=4, dt=0.02)
    o.set_f(np.zeros((n, 65)))
    x = np.linspace(-2, 2, n)
    k = 2.0
    o.push_frozen(-np.sin(k * x), -k * np.cos(k * x), k * k * np.sin(k * x), 0.0, 0.0, 30)
    o.compute_map()
    assert o.diagnostics()["emap"] > 1e-6


def test_gaussian_initial_condition_mass_and_cut():
    """The paper's Gaussian IC (Sec. 3.2): total mass rho 2 pi sigma^2
    (1 - exp(-R^2 / 2 sigma^2)) plus a negligible apodised rim, continuous
    at R, zero beyond R + eta atanh(1/2)."""
    p = {"rho": 4.0, "sigma": 0.2, "R": 1.0, "eta": 0.02}
    n = 1201
    x = np.linspace(-1.2, 1.2, n)
    X, V = np.meshgrid(x, x, indexing="ij")
    f = I.gaussian_ic(X, V, **p)
    dx = x[1] - x[0]
    exact = p["rho"] * 2 * math.pi * p["sigma"] ** 2 * (1 - math.exp(-p["R"] ** 2 / (2 * p["sigma"] ** 2)))
    assert f.sum() * dx * dx == pytest.approx(exact, rel=1e-6)
    r_cut = p["R"] + p["eta"] * math.atanh(0.5)
    assert I.gaussian_ic(p["R"], 0.0, **p) == pytest.approx(I.gaussian_ic(p["R"] - 1e-12, 0.0, **p), rel=1e-9)
    assert I.gaussian_ic(r_cut + 1e-9, 0.0, **p) == 0.0 and I.gaussian_ic(r_cut - 1e-3, 0.0, **p) > 0.0


def test_variable_time_step_follows_the_density_constraint():
    """Sec. 2.4: Delta t = min(dt, C_dyn / sqrt(rho_max)).  For the isothermal
    sheet rho(x) = rho_0 sech^2(x / x_0), rho_0 = 2 pi (M = 1, G = 1, sigma =
    1/2); the grid has no node at x = 0, so rho_max is rho at x = +-dx/2.  A
    large C_dyn leaves the constant step."""
    rc = I.SPITZER_128
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_f(I.initial_f(rc))
    c = 0.005
    o.set_cdyn(c)
    o.step(1)
    x0 = 0.25 / math.pi
    rho_max = 2 * math.pi / math.cosh(0.5 * rc.dx / x0) ** 2
    assert o.last_dt() == pytest.approx(c / math.sqrt(rho_max), rel=1e-4)
    assert o.time() == pytest.approx(o.last_dt(), rel=1e-15)
    big = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    plain = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    for z in (big, plain):
        z.set_f(I.initial_f(rc))
    big.set_cdyn(1e6)
    big.step(3)
    plain.step(3)
    assert big.last_dt() == rc.dt and big.time() == pytest.approx(3 * rc.dt)
    assert np.array_equal(big.elements(), plain.elements())
