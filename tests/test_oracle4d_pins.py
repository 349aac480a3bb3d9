"""Pins of the FP64 oracle of the 4D phase-space step against closed forms,
invariants and brute force (no GPU).

Each test fixes one piece against something other than the oracle itself:
the 15-point quadratic hypersurface of Sec. 2.2.1 (exact on every quadratic
in all 16 orthants), the tensor-product spline of Sec. 2.2.2 (a dense
Kronecker solve), the inverse map of Sec. 2.1 (exact for H = 0, third order
otherwise), the beta set of Sec. 2.3.2 (it holds every element the kernel
support reaches), the percolation of Sec. 2.3.1 (nearest lattice element
after a remap; connected components by scipy labelling on a distorted
state), the Poisson field of Sec. 2.5 in 2D space (the closed-form field of
a Gaussian disc, Newton's third law), the element push of Sec. 2.4 (the
linear leapfrog matrix; T and H against finite differences of trajectories),
free streaming (G = 0) against the interpolation of f0 at the exact
characteristics, and Q_r on hand-built displaced elements.
"""
import itertools
import math

import numpy as np
import pytest

import oracle.oracle as O2
import oracle.oracle4d as Q
from paper_1705_03750_gb300 import inputs4d as I4

RNG = np.random.default_rng(20240)


# ---- Sec. 2.2.1: 15-point quadratic interpolation --------------------------

def _quad(coef, X):
    """c0 + sum_a c_a x_a + sum_{a<=b} c_ab x_a x_b on points X[..., 4]."""
    v = coef[0] + sum(coef[1 + a] * X[..., a] for a in range(4))
    k = 5
    for a in range(4):
        for b in range(a, 4):
            v = v + coef[k] * X[..., a] * X[..., b]
            k += 1
    return v


def test_qinterp_exact_on_quadratics_in_every_orthant():
    n = (7, 6, 8, 7)
    idx = np.stack(np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij"), axis=-1)
    for _ in range(4):
        coef = RNG.normal(size=15)
        F = _quad(coef, idx)
        for signs in itertools.product((-1, 1), repeat=4):
            u = np.array([3.0, 2.0, 4.0, 3.0]) + np.array(signs) * RNG.uniform(0.05, 0.49, 4)
            assert Q.qinterp(F, u) == pytest.approx(_quad(coef, u), abs=1e-11)


def test_qinterp_passes_through_its_15_nodes_and_only_uses_them():
    n = (6, 6, 6, 6)
    F = RNG.normal(size=n)
    # at a node the value is the node's
    assert Q.qinterp(F, [2.0, 3.0, 1.0, 4.0]) == pytest.approx(F[2, 3, 1, 4], abs=1e-14)
    u = np.array([2.3, 2.8, 3.1, 2.6])           # nearest (2, 3, 3, 3); dq signs + - + -
    base = Q.qinterp(F, u)
    used = set()
    gn = (2, 3, 3, 3)
    used.add(gn)
    for a in range(4):
        for s in (-1, 1):
            g = list(gn)
            g[a] += s
            used.add(tuple(g))
    gc = np.floor(u).astype(int)
    for a in range(4):
        for b in range(a + 1, 4):
            g = list(gn)
            g[a] = gc[a] + 1 if gc[a] == gn[a] else gc[a]
            g[b] = gc[b] + 1 if gc[b] == gn[b] else gc[b]
            used.add(tuple(g))
    assert len(used) == 15
    for g in itertools.product(*[range(k) for k in n]):
        G = F.copy()
        G[g] += 1.0
        changed = Q.qinterp(G, u) != base
        assert changed == (g in used), g


def test_qinterp_reads_zero_outside_the_grid():
    F = np.ones((5, 5, 5, 5))
    # beyond the range the value is 0; at an edge the missing neighbour reads 0
    assert Q.qinterp(F, [-2.5, 2, 2, 2]) == 0.0
    assert Q.qinterp(F, [4.0, 2, 2, 2]) == pytest.approx(1.0)
    v = Q.qinterp(F, [4.3, 2, 2, 2])             # nearest 4, F(5) = 0: 1 - dq^2 + dq(dq-1)/2
    dq = 0.3
    assert v == pytest.approx((1 - dq * dq) + 0.5 * dq * (dq - 1.0), abs=1e-14)


# ---- Sec. 2.2.2: tensor-product cubic spline ---------------------------------

def _spline_matrix(n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = 4.0
        if i > 0:
            A[i, i - 1] = 1.0
        if i < n - 1:
            A[i, i + 1] = 1.0
    A[0, 1] = 2.0
    A[n - 1, n - 2] = 2.0
    return A / 6.0


def test_spline_solve_matches_a_dense_kronecker_solve():
    n = (5, 4, 6, 5)
    f = RNG.normal(size=n)
    K = _spline_matrix(n[0])
    for a in range(1, 4):
        K = np.kron(K, _spline_matrix(n[a]))
    ref = np.linalg.solve(K, f.ravel()).reshape(n)
    np.testing.assert_allclose(Q.spline_solve(f), ref, atol=1e-12, rtol=0)


def test_spline_reproduces_nodes_and_a_bump_has_a_unit_coefficient():
    n = (8, 7, 9, 8)
    f = RNG.normal(size=n)
    eta = Q.spline_solve(f)
    for g in [(0, 0, 0, 0), (3, 2, 4, 5), (7, 6, 8, 7), (1, 5, 0, 3)]:
        assert Q.spline_eval(eta, np.array(g, float)) == pytest.approx(f[g], abs=1e-12)
    # an interior bump B(u-k)... sampled on the nodes has eta = unit vector
    k = (3, 3, 4, 4)
    b = [np.array([O2.bspline3(i - k[a]) for i in range(n[a])]) for a in range(4)]
    fb = np.einsum("i,j,k,l->ijkl", *b)
    e = Q.spline_solve(fb)
    unit = np.zeros(n)
    unit[k] = 1.0
    np.testing.assert_allclose(e, unit, atol=1e-12)
    u = np.array([3.3, 2.6, 4.7, 3.9])
    ref = np.prod([O2.bspline3(u[a] - k[a]) for a in range(4)])
    assert Q.spline_eval(e, u) == pytest.approx(ref, abs=1e-13)


# ---- Sec. 2.1: inverse map ---------------------------------------------------

def _elem(P, T, H):
    return np.concatenate([P, T.ravel(), H.ravel()])


def _sym10(Hfull):
    """H[a][b][c] -> 4 x 10 in the order 00,01,02,03,11,12,13,22,23,33."""
    out = np.zeros((4, 10))
    k = 0
    for b in range(4):
        for c in range(b, 4):
            out[:, k] = Hfull[:, b, c]
            k += 1
    return out


def _random_T():
    return np.eye(4) + 0.3 * RNG.normal(size=(4, 4))


def test_taylor_inverse_matches_numpy():
    for _ in range(10):
        T = _random_T()
        t = Q.taylor_one(_elem(np.zeros(4), T, np.zeros((4, 10))), np.zeros(4))
        np.testing.assert_allclose(t[4:20].reshape(4, 4), np.linalg.inv(T), rtol=0, atol=1e-13)


def test_inverse_map_exact_for_linear_and_third_order_for_quadratic():
    T = _random_T()
    Pm = RNG.normal(size=4)
    Qm = RNG.normal(size=4)
    t = Q.taylor_one(_elem(Pm, T, np.zeros((4, 10))), Qm)
    dQ = RNG.normal(size=4) * 0.3
    P = Pm + T @ dQ
    np.testing.assert_allclose(Q.qofp(t, P), dQ, atol=1e-14)
    # quadratic forward map P = Pm + T dQ + H(dQ, dQ)/2 with symmetric H
    Hf = RNG.normal(size=(4, 4, 4))
    Hf = 0.5 * (Hf + Hf.transpose(0, 2, 1))
    t = Q.taylor_one(_elem(Pm, T, _sym10(Hf)), Qm)
    d0 = RNG.normal(size=4)
    d0 /= np.linalg.norm(d0)
    errs = []
    for h in (0.02, 0.01, 0.005):
        dq = h * d0
        P = Pm + T @ dq + 0.5 * np.einsum("abc,b,c->a", Hf, dq, dq)
        errs.append(np.linalg.norm(Q.qofp(t, P) - dq))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, (errs, r1, r2)


# ---- Sec. 2.3: ranges ------------------------------------------------------

def test_alpha_offsets_cover_the_closer_lattice_neighbours():
    assert Q.alpha_offsets([0.1, -0.2, 0.3, -0.4]) == []
    assert len(Q.alpha_offsets([0.45, -0.45, 0.45, -0.45])) == 15
    # one axis beyond alpha: the single neighbour on that side
    assert Q.alpha_offsets([0.0, 0.0, -0.44, 0.0]) == [(0, 0, -1, 0)]


def test_beta_set_holds_every_neighbour_the_kernel_reaches():
    # W(2 d) > 0 needs d < 1: on the undistorted lattice the offsets o with
    # |xi - o| < 1 from a point in the owner's cell must all be in the set
    for _ in range(3000):
        xi = RNG.uniform(-0.5, 0.5, 4)
        got = set(Q.beta_offsets(xi))
        for o in itertools.product((-1, 0, 1), repeat=4):
            if np.sum((xi - np.array(o)) ** 2) < 1.0:
                assert o in got, (xi, o)
    assert len(Q.beta_offsets([0, 0, 0, 0])) == 9
    assert len(Q.beta_offsets([0.3, 0.3, -0.3, 0.3])) == 16
    # the 2D rule of the paper on the (x, vx) plane when y, vy sit far out
    got = Q.beta_offsets([0.0, 0.3, 0.2, 0.3])
    assert (1, 0, 1, 0) not in got and (0, 1, 0, 1) in got


# ---- Sec. 2.3.1: percolation map --------------------------------------------

def test_map_after_reset_is_the_nearest_lattice_element():
    rc = I4.HALOS4D_16.with_(n=(16, 12, 14, 10))
    o = Q.Oracle4D.from_run(rc)
    o.set_f(np.zeros(rc.n))
    m, st = o.compute_map()
    assert st == 0
    L = o.Ldims
    d = rc.d
    ks = []
    for a in range(4):
        K = (L[a] - 3) // 2
        ctr = 0.5 * (rc.lo[a] + rc.hi[a])
        x = rc.axis(a)
        k = np.floor((x - ctr) / (rc.s * d[a]) + 0.5).astype(int) + K + 1
        ks.append(k)
    ref = ((ks[0][:, None, None, None] * L[1] + ks[1][None, :, None, None]) * L[2]
           + ks[2][None, None, :, None]) * L[3] + ks[3][None, None, None, :]
    assert (m == ref).all()


def _np_taylor(o):
    return o.taylor()


def _d2_all(t, P, inv_dm):
    """d^2 of one Taylor record at the sites P[..., 4], in the oracle's order."""
    dP = [P[..., a] - t[a] for a in range(4)]
    Ti = t[4:20]
    y = [((Ti[4 * a] * dP[0] + Ti[4 * a + 1] * dP[1]) + Ti[4 * a + 2] * dP[2]) + Ti[4 * a + 3] * dP[3]
         for a in range(4)]
    sy = [[0, 1, 2, 3], [1, 4, 5, 6], [2, 5, 7, 8], [3, 6, 8, 9]]
    s = []
    for l in range(4):
        G = t[20 + 10 * l:30 + 10 * l]
        g = [((G[sy[b][0]] * dP[0] + G[sy[b][1]] * dP[1]) + G[sy[b][2]] * dP[2]) + G[sy[b][3]] * dP[3]
             for b in range(4)]
        s.append(((dP[0] * g[0] + dP[1] * g[1]) + dP[2] * g[2]) + dP[3] * g[3])
    x = []
    for a in range(4):
        c = ((Ti[4 * a] * s[0] + Ti[4 * a + 1] * s[1]) + Ti[4 * a + 2] * s[2]) + Ti[4 * a + 3] * s[3]
        x.append((y[a] - 0.5 * c) * inv_dm[a])
    return ((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]) + x[3] * x[3], x


def test_map_components_match_scipy_labelling_on_a_distorted_state():
    ndimage = pytest.importorskip("scipy.ndimage")
    rc = I4.HALOS4D_16.with_(n=(7, 6, 7, 6), s=3)
    o = Q.Oracle4D.from_run(rc)
    o.set_f(np.zeros(rc.n))
    el = o.elements()
    # distort: random T near I, small H, displaced positions
    rng = np.random.default_rng(7)
    for m in range(o.ne):
        T = np.eye(4) + 0.15 * rng.normal(size=(4, 4))
        el[m, 4:20] = T.ravel()
        el[m, 20:60] = 0.3 * rng.normal(size=40)
        el[m, 0:4] += 0.2 * rng.normal(size=4) * np.array(rc.d) * rc.s
    o.set_elements(el)
    m_or, st = o.compute_map()
    assert st == 0
    assert o.map_stats()["multi_claims"] > 0      # overlapping components occur
    tay = o.taylor()
    pad = rc.s
    n = np.array(rc.n)
    grids = [rc.lo[a] + np.arange(-pad, n[a] + pad) * rc.d[a] for a in range(4)]
    P = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1)
    inv_dm = [1.0 / (rc.s * rc.d[a]) for a in range(4)]
    Ld = o.Ldims
    D = np.stack([_d2_all(tay[m], P, inv_dm)[0] for m in range(o.ne)])
    best = np.full(rc.n, np.inf)
    owner = np.full(rc.n, -1, dtype=np.int64)
    alpha = Q.ALPHA
    struct = ndimage.generate_binary_structure(4, 1)
    for m in range(o.ne):
        k = np.unravel_index(m, Ld)
        g0 = [int(math.floor((el[m, a] - rc.lo[a]) / rc.d[a] + 0.5)) for a in range(4)]
        if any(g0[a] < -pad or g0[a] >= n[a] + pad for a in range(4)):
            continue
        d2, x = _d2_all(tay[m], P, inv_dm)
        ok = np.ones(d2.shape, bool)
        lo = [np.where(x[a] < -alpha, -1, 0) for a in range(4)]
        hi = [np.where(x[a] < alpha, 0, 1) for a in range(4)]
        hi = [np.where(x[a] < -alpha, 0, hi[a]) for a in range(4)]
        for off in itertools.product((-1, 0, 1), repeat=4):
            if off == (0, 0, 0, 0):
                continue
            kk = [k[a] + off[a] for a in range(4)]
            if any(kk[a] < 0 or kk[a] >= Ld[a] for a in range(4)):
                continue
            inr = np.ones(d2.shape, bool)
            for a in range(4):
                inr &= (lo[a] <= off[a]) & (off[a] <= hi[a])
            ok &= ~(inr & (D[np.ravel_multi_index(kk, Ld)] < d2))
        lab, _ = ndimage.label(ok, structure=struct)
        l0 = lab[tuple(g0[a] + pad for a in range(4))]
        if l0 == 0:
            continue
        comp = (lab == l0)[pad:pad + n[0], pad:pad + n[1], pad:pad + n[2], pad:pad + n[3]]
        dd = d2[pad:pad + n[0], pad:pad + n[1], pad:pad + n[2], pad:pad + n[3]]
        better = comp & ((dd < best) | ((dd == best) & (m < owner)))
        best[better] = dd[better]
        owner[better] = m
    # holes: Jacobi rounds over the 8 face neighbours
    Pin = P[pad:pad + n[0], pad:pad + n[1], pad:pad + n[2], pad:pad + n[3]]
    rounds = 0
    while (owner < 0).any():
        prev = owner.copy()
        for g in zip(*np.nonzero(prev < 0)):
            cand = []
            for a in range(4):
                for s_ in (-1, 1):
                    h = list(g)
                    h[a] += s_
                    if 0 <= h[a] < n[a] and prev[tuple(h)] >= 0:
                        c = int(prev[tuple(h)])
                        d2c, _ = _d2_all(tay[c], Pin[g], inv_dm)
                        cand.append((float(d2c), c))
            if cand:
                owner[g] = min(cand)[1]
        rounds += 1
        assert rounds < 50
    assert (owner == m_or).all(), int((owner != m_or).sum())


# ---- Sec. 2.5: Poisson in 2D space ------------------------------------------

def test_field_of_a_gaussian_disc_converges_to_the_closed_form():
    # rho = M/(2 pi s^2) exp(-r^2/2s^2): g(r) = -2 G M (1 - exp(-r^2/2s^2)) / r
    G, M, sg = 1.0, 1.0, 0.2
    errs = []
    for n in (33, 65):
        x = np.linspace(-1, 1, n)
        dx = x[1] - x[0]
        X, Y = np.meshgrid(x, x, indexing="ij")
        Mp = M / (2 * math.pi * sg * sg) * np.exp(-(X * X + Y * Y) / (2 * sg * sg)) * dx * dx
        e = 0.0
        for (i, j) in [(n // 2 + n // 8, n // 2), (n // 2 + n // 4, n // 2 - n // 8),
                       (n // 2 - n // 4, n // 2 + n // 4)]:
            g = Q.accel_at_node(Mp, dx, dx, G, i, j)
            r = np.array([x[i], x[j]])
            rr = np.linalg.norm(r)
            ref = -2 * G * M * (1 - math.exp(-rr * rr / (2 * sg * sg))) / rr * r / rr
            e = max(e, np.abs(g - ref).max())
        errs.append(e)
    assert errs[1] < 0.3 * errs[0] and errs[1] < 0.02, errs  # second order in dx


def test_field_obeys_newtons_third_law_and_the_far_field():
    Mp = RNG.uniform(0, 1, size=(6, 5))
    dx, dy, G = 0.1, 0.12, 0.7
    F = sum(Mp[i, j] * Q.accel_at_node(Mp, dx, dy, G, i, j) for i in range(6) for j in range(5))
    assert np.abs(F).max() < 1e-12
    # far from the grid the field is that of the total mass at the centre of mass
    i, j = 4000, -3000
    g = Q.accel_at_node(Mp, dx, dy, G, i, j)
    cm = np.array([(Mp.sum(1) * np.arange(6)).sum(), (Mp.sum(0) * np.arange(5)).sum()]) / Mp.sum()
    r = np.array([(i - cm[0]) * dx, (j - cm[1]) * dy])
    ref = -2 * G * Mp.sum() * r / (r @ r)
    np.testing.assert_allclose(g, ref, rtol=1e-6)


def test_field_derivatives_are_the_centred_differences_of_an_exact_field():
    # a single pixel mass: g = -2 G m r/|r|^2 at every other node; J and K
    # against the analytic derivatives at O(dx^2) far from the mass
    Mp = np.zeros((41, 41))
    Mp[20, 20] = 1.0
    dx = 0.05
    out = Q.field_at_node(Mp, dx, dx, 1.0, 40, 30)
    x, y = 20 * dx, 10 * dx
    r2 = x * x + y * y
    gx, gy = -2 * x / r2, -2 * y / r2
    Jxx = -2 * (r2 - 2 * x * x) / r2 ** 2
    Jxy = 4 * x * y / r2 ** 2
    Jyy = -2 * (r2 - 2 * y * y) / r2 ** 2
    assert out[0] == pytest.approx(gx, rel=1e-12) and out[1] == pytest.approx(gy, rel=1e-12)
    np.testing.assert_allclose(out[2:6], [Jxx, Jxy, Jxy, Jyy], rtol=2e-2)
    # Kx_xx = d2 gx/dx2 analytic
    Kxxx = -2 * (2 * x ** 3 - 6 * x * y * y) / r2 ** 3
    assert out[6] == pytest.approx(Kxxx, rel=5e-2)


# ---- Sec. 2.4: element push -------------------------------------------------

def test_linear_force_gives_the_leapfrog_matrix():
    rc = I4.HALOS4D_16.with_(n=(8, 8, 8, 8), s=4, dt=0.05)
    o = Q.Oracle4D.from_run(rc)
    o.set_f(np.zeros(rc.n))
    A = np.array([[-1.0, 0.3], [0.3, -2.0]])
    coef = np.concatenate([[0.0, 0.0], A.ravel(), np.zeros(6)])
    el0 = o.elements()
    o.push_frozen(coef, 7)
    el = o.elements()
    h = 0.5 * rc.dt
    D = np.eye(4)
    D[0, 2] = D[1, 3] = h
    K = np.eye(4)
    K[2:, :2] = A * rc.dt
    Mstep = D @ K @ D
    Mn = np.linalg.matrix_power(Mstep, 7)
    for m in (0, 100, 400, o.ne - 1):
        np.testing.assert_allclose(el[m, 4:20].reshape(4, 4), Mn, atol=1e-13)
        np.testing.assert_allclose(el[m, 0:4], Mn @ el0[m, 0:4], atol=1e-13)
        assert np.abs(el[m, 20:]).max() < 1e-12   # second differences of a linear field
    assert np.linalg.det(Mn) == pytest.approx(1.0, abs=1e-13)


def test_quadratic_force_T_and_H_match_finite_differences_of_trajectories():
    rc = I4.HALOS4D_16.with_(n=(8, 8, 8, 8), s=4, dt=0.04)
    d = rc.d
    o = Q.Oracle4D.from_run(rc)
    o.set_f(np.zeros(rc.n))
    c = np.array([0.1, -0.2])
    A = np.array([[-1.0, 0.4], [0.2, -1.5]])
    B = np.array([[0.8, -0.3, 0.5], [-0.6, 0.7, 0.2]])  # xx, xy, yy per component
    coef = np.concatenate([c, A.ravel(), B.ravel()])
    steps = 6
    el0 = o.elements()
    o.push_frozen(coef, steps)
    el = o.elements()
    # TSC of a quadratic adds the constant B_xx dx^2/8 + B_yy dy^2/8 to g;
    # the differences of a quadratic are exact
    off = np.array([B[a, 0] * d[0] ** 2 / 8 + B[a, 2] * d[1] ** 2 / 8 for a in range(2)])

    def g(x, y):
        return np.array([c[a] + A[a, 0] * x + A[a, 1] * y
                         + 0.5 * (B[a, 0] * x * x + 2 * B[a, 1] * x * y + B[a, 2] * y * y)
                         for a in range(2)]) + off

    def traj(q):
        p = q.astype(float).copy()
        for _ in range(steps):
            p[:2] += 0.5 * rc.dt * p[2:]
            p[2:] += rc.dt * g(p[0], p[1])
            p[:2] += 0.5 * rc.dt * p[2:]
        return p

    for m in (5, 300, 600):
        q = el0[m, :4]
        np.testing.assert_allclose(el[m, :4], traj(q), atol=1e-12)
        hh = 1e-3
        Tfd = np.zeros((4, 4))
        Hfd = np.zeros((4, 4, 4))
        for b in range(4):
            eb = np.eye(4)[b] * hh
            Tfd[:, b] = (traj(q + eb) - traj(q - eb)) / (2 * hh)
            for cc in range(4):
                ec = np.eye(4)[cc] * hh
                Hfd[:, b, cc] = (traj(q + eb + ec) - traj(q + eb - ec) - traj(q - eb + ec)
                                 + traj(q - eb - ec)) / (4 * hh * hh)
        np.testing.assert_allclose(el[m, 4:20].reshape(4, 4), Tfd, atol=1e-8)
        np.testing.assert_allclose(el[m, 20:60].reshape(4, 10), _sym10(Hfd), atol=2e-5)


# ---- whole method -----------------------------------------------------------

def test_free_streaming_is_the_interpolation_at_the_exact_characteristics():
    rc = I4.FREE4D_16.with_(n_s=3)
    o = Q.Oracle4D.from_run(rc)
    f0 = I4.initial_f4(rc)
    o.set_f(f0)
    o.step(2)                         # f(t + dt/2) of step 2: t = 1.5 dt
    f = o.last_f()
    t = 1.5 * rc.dt
    d = rc.d
    for g in [(3, 4, 7, 9), (8, 8, 8, 8), (12, 2, 5, 11), (0, 15, 14, 1)]:
        P = np.array([rc.lo[a] + g[a] * d[a] for a in range(4)])
        Qx = P[:2] - P[2:] * t
        u = [(Qx[0] - rc.lo[0]) / d[0], (Qx[1] - rc.lo[1]) / d[1], g[2], g[3]]
        assert f[g] == pytest.approx(Q.qinterp(f0, u), abs=1e-13 * f0.max())
    # through the remap (end of step 3): f_ini = spline of f0 at the exact Q
    o.step(1)
    fi = o.fini()
    eta0 = Q.spline_solve(f0)
    t = 3 * rc.dt
    for g in [(3, 4, 7, 9), (8, 8, 8, 8), (12, 2, 5, 11)]:
        P = np.array([rc.lo[a] + g[a] * d[a] for a in range(4)])
        Qx = P[:2] - P[2:] * t
        u = [(Qx[0] - rc.lo[0]) / d[0], (Qx[1] - rc.lo[1]) / d[1], g[2], g[3]]
        assert fi[g] == pytest.approx(Q.spline_eval(eta0, u), abs=1e-13 * f0.max())


def test_blended_q_on_displaced_isotropic_elements():
    # T = I, H = 0, element m' displaced by e_m': Q(P, m') = Q_m' + P - P_m' =
    # P - e_m'; Q_r = sum W(2 d) (P - e) / sum W(2 d), d = |P - e - Q_m'| in
    # element spacings
    rc = I4.HALOS4D_16.with_(n=(12, 12, 12, 12), s=4)
    o = Q.Oracle4D.from_run(rc)
    o.set_f(np.zeros(rc.n))
    el = o.elements()
    rng = np.random.default_rng(3)
    dm = np.array(rc.d) * rc.s
    disp = 0.05 * rng.normal(size=(o.ne, 4)) * dm
    lat = el[:, :4].copy()
    el[:, :4] += disp
    o.set_elements(el)
    _, Qr = o.remap_resample()
    owner, _ = o.compute_map()
    for g in [(5, 6, 5, 6), (4, 7, 6, 5), (6, 5, 7, 4), (2, 9, 3, 8)]:
        P = np.array([rc.lo[a] + g[a] * rc.d[a] for a in range(4)])
        m = owner[g]
        xi = (P - disp[m] - lat[m]) / dm
        k = np.unravel_index(m, o.Ldims)
        num, den = np.zeros(4), 0.0
        for off in Q.beta_offsets(xi):
            kk = [k[a] + off[a] for a in range(4)]
            mm = np.ravel_multi_index(kk, o.Ldims)
            dd = np.linalg.norm((P - disp[mm] - lat[mm]) / dm)
            w = O2.W(2 * dd)
            num += w * (P - disp[mm])
            den += w
        np.testing.assert_allclose(Qr[g], num / den, atol=1e-14)
        # and a plausible slip (the weight of d instead of 2d) differs
        num2, den2 = np.zeros(4), 0.0
        for off in Q.beta_offsets(xi):
            kk = [k[a] + off[a] for a in range(4)]
            mm = np.ravel_multi_index(kk, o.Ldims)
            dd = np.linalg.norm((P - disp[mm] - lat[mm]) / dm)
            num2 += O2.W(dd) * (P - disp[mm])
            den2 += O2.W(dd)
        assert np.abs(num2 / den2 - Qr[g]).max() > 1e-6


def test_mass_is_conserved_to_interpolation_accuracy_and_det_T_stays_one():
    rc = I4.HALOS4D_16
    o = Q.Oracle4D.from_run(rc)
    f0 = I4.initial_f4(rc)
    o.set_f(f0)
    m0 = f0.sum() * np.prod(rc.d)
    o.step(3)
    dg = o.diagnostics()
    assert abs(dg["mass"] - m0) < 2e-3
    assert abs(dg["detT_min"] - 1) < 1e-4 and abs(dg["detT_max"] - 1) < 1e-4


def _centred_halo(rc):
    x = [rc.axis(a) for a in range(4)]
    X = np.meshgrid(*x, indexing="ij")
    f0 = np.exp(-0.5 * ((X[0] / 0.3) ** 2 + (X[1] / 0.25) ** 2 + (X[2] / 0.35) ** 2 + (X[3] / 0.3) ** 2))
    return f0 / (f0.sum() * np.prod(rc.d))


def test_point_symmetry_is_kept_through_a_remap():
    # an IC symmetric under P -> -P on a box and lattice centred at 0 stays
    # symmetric (a mirrored stencil, axis or index slip would break it)
    rc = I4.HALOS4D_16
    o = Q.Oracle4D.from_run(rc)
    f0 = _centred_halo(rc)
    o.set_f(f0)
    for _ in range(rc.n_s + 1):
        o.step(1)
        f = o.last_f()
        assert np.abs(f - f[::-1, ::-1, ::-1, ::-1]).max() <= 1e-12 * f.max()


def test_a_halo_at_rest_falls_in_and_conserves_energy():
    # gravity attracts: kinetic energy rises and potential energy falls; the
    # total holds to the scheme's accuracy on this coarse grid (its mass
    # moves by a few 1e-4 through the remap)
    rc = I4.HALOS4D_16
    o = Q.Oracle4D.from_run(rc)
    o.set_f(_centred_halo(rc))
    d0 = o.diagnostics()
    o.step(rc.n_s + 1)
    d1 = o.diagnostics()
    assert d1["ekin"] > d0["ekin"] * 1.005 and d1["epot"] < d0["epot"] - 1e-3
    e0, e1 = d0["ekin"] + d0["epot"], d1["ekin"] + d1["epot"]
    assert abs(e1 - e0) < 1e-3 * abs(e0)
