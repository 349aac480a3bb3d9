"""Pins of the oracle's smooth map Q_r (Sec. 2.3.2, eq. interpol) and of its
E_map estimate (Sec. 2.3.2, last subsection) on hand-built states.

Isotropic elements (T = I, H = 0) whose anchors P_m are displaced from their
lattice positions Q_m by known vectors delta_m propose, at any site P,
Q(P, m) = P - delta_m exactly, at the distance d_m = |P - P_m| in element
spacings.  Choosing the displacements so that every distance is a simple
fraction makes Q_r a weighted mean that can be worked out by hand, with the
Monaghan kernel evaluated at 2d in {0.5, 1, 1.5} (W = 23/32, 1/4, 1/32).
The expected values below are those hand results, written out as
fractions; a kernel evaluated at d instead of 2d, an unnormalised sum, a
dropped owner term, a diagonal kept where the paper's cross rule drops it,
or the other element's proposal all give different numbers.

For the same kind of state the mismatch that E_map measures between the
owner m and a neighbour n, ((a + xi_n) - xi_m, (b + ze_n) - ze_m), is
delta_m - delta_n in element spacings, whatever the site: with a single
displaced element E_map is |delta| (Euclidean norm, element units).
"""
import math

import numpy as np
import pytest

import oracle.oracle as O

# 65 x 65 nodes on [-2, 2]^2 (dx = dv = 1/16), elements every 4 sites
# (spacing 1/4), lattice index 9 at the centre of the box.
N, S, BOX = 65, 4, (-2.0, 2.0, -2.0, 2.0)
DM = S * (BOX[1] - BOX[0]) / (N - 1)   # element spacing, both axes


def _lattice_oracle(nx=N, nv=N, box=BOX, s=S):
    o = O.Oracle(nx, nv, box[0], box[1], box[2], box[3], s, 0.01, 1000, 0.0)
    o.set_f(np.zeros((nx, nv)))
    return o


def _displace(o, moves, dxm, dvm):
    """Move the anchors of the elements (k, l) by delta (element units)."""
    el = o.elements()
    for (k, l), (ax, av) in moves.items():
        m = k * o.Lv + l
        el[m, 0] += ax * dxm
        el[m, 1] += av * dvm
    o.set_elements(el)


def _node(o, x, v):
    i = round((x - BOX[0]) / o.dx)
    j = round((v - BOX[2]) / o.dv)
    assert abs(BOX[0] + i * o.dx - x) < 1e-15 and abs(BOX[2] + j * o.dv - v) < 1e-15
    return i, j


def _q_lattice(o, k, l, box=BOX, dxm=DM, dvm=DM):
    Kx = (o.Lx - 3) // 2
    Kv = (o.Lv - 3) // 2
    return 0.5 * (box[0] + box[1]) + (k - Kx - 1) * dxm, 0.5 * (box[2] + box[3]) + (l - Kv - 1) * dvm


# Owner (9, 9) at Q = (0, 0), anchor moved by (0.1, 0.05); the site sits at
# (1/4, 1/4) of an element spacing from Q, so P - P_m = (0.15, 0.2), d = 1/4,
# and both offsets exceed beta: the 2 x 2 set {(0,0), (1,0), (0,1), (1,1)}.
#   (10, 9) moved by (0.3, 0):     P - P_n = (-1.05, 0.25), d > 1/2 (weight 0)
#   (9, 10) moved by (0, 0.3):     P - P_n = (0.25, -1.05), d > 1/2 (weight 0)
#   (10, 10) moved by (-.45, -.35): P - P_n = (-0.3, -0.4),  d = 1/2, W(1) = 1/4
# Q_r - P = [23/32 (-0.1, -0.05) + 1/4 (0.45, 0.35)] / (31/32) = (13/310, 33/620)
QUADRANT = {(9, 9): (0.1, 0.05), (10, 9): (0.3, 0.0), (9, 10): (0.0, 0.3), (10, 10): (-0.45, -0.35)}
QUADRANT_SITE = (0.25, 0.25)
QUADRANT_QR = (13 / 310, 33 / 620)

# Owner (5, 5) at Q = (-1, -1), not moved; the site is Q itself, so xi = ze = 0:
# both axes take {-1, 0, 1} and only the cross survives.
#   (6, 5) moved by (-0.25, 0): P - P_n = (-0.75, 0), d = 3/4, W(3/2) = 1/32
#   (5, 4) moved by (0, 0.5):   P - P_n = (0, 0.5),   d = 1/2, W(1)   = 1/4
#   (6, 6) moved by (-0.6, -0.7): d = 1/2 too, but it is a diagonal: dropped
# Q_r - P = [1/32 (0.25, 0) + 1/4 (0, -0.5)] / (41/32) = (1/164, -4/41)
CROSS = {(6, 5): (-0.25, 0.0), (5, 4): (0.0, 0.5), (6, 6): (-0.6, -0.7)}
CROSS_QR = (1 / 164, -4 / 41)


def _qr_state():
    o = _lattice_oracle()
    _displace(o, {**QUADRANT, **CROSS}, DM, DM)
    fnew, qr = o.remap_resample()
    m, _ = o.compute_map()
    return o, qr, m


def test_blended_map_quadrant_case_by_hand():
    o, qr, owner = _qr_state()
    qx, qv = _q_lattice(o, 9, 9)
    Px, Pv = qx + QUADRANT_SITE[0] * DM, qv + QUADRANT_SITE[1] * DM
    i, j = _node(o, Px, Pv)
    assert owner[i, j] == 9 * o.Lv + 9
    got = (qr[i, j, 0] - Px) / DM, (qr[i, j, 1] - Pv) / DM
    assert got == pytest.approx(QUADRANT_QR, abs=1e-13)
    # plausible slips give other numbers: the owner's proposal alone, the
    # kernel at d, an unnormalised sum
    assert abs(got[0] - (-0.1)) > 0.1
    w_d = [1 - 1.5 * 0.25 ** 2 + 0.75 * 0.25 ** 3, 1 - 1.5 * 0.5 ** 2 + 0.75 * 0.5 ** 3]
    slip = (w_d[0] * -0.1 + w_d[1] * 0.45) / (w_d[0] + w_d[1])
    assert abs(got[0] - slip) > 1e-2
    assert abs(got[0] - 13 / 320) > 1e-3


def test_blended_map_cross_case_by_hand():
    o, qr, owner = _qr_state()
    Px, Pv = _q_lattice(o, 5, 5)
    i, j = _node(o, Px, Pv)
    assert owner[i, j] == 5 * o.Lv + 5
    got = (qr[i, j, 0] - Px) / DM, (qr[i, j, 1] - Pv) / DM
    assert got == pytest.approx(CROSS_QR, abs=1e-13)
    # with the diagonal (6, 6) kept, its weight 1/4 and proposal (0.6, 0.7)
    # would move Q_r by more than 0.1 of an element spacing
    with_diag = ((1 / 128 + 0.15), (-1 / 8 + 0.175))
    assert abs(got[1] - with_diag[1] / (41 / 32 + 1 / 4)) > 0.05


def test_blended_map_is_the_owner_map_where_no_neighbour_reaches():
    """Away from every displaced element the lattice is untouched: each site
    gets Q_r = P (all proposals equal P there)."""
    o, qr, owner = _qr_state()
    X, V = np.meshgrid(np.linspace(*BOX[:2], N), np.linspace(*BOX[2:], N), indexing="ij")
    far = (np.abs(X - 1.25) < 0.3) & (np.abs(V - 1.25) < 0.3)
    np.testing.assert_allclose(qr[far, 0], X[far], atol=1e-14)
    np.testing.assert_allclose(qr[far, 1], V[far], atol=1e-14)


def _emap_of(moves, nx=N, nv=N, box=BOX, s=S):
    o = _lattice_oracle(nx, nv, box, s)
    dxm = s * (box[1] - box[0]) / (nx - 1)
    dvm = s * (box[3] - box[2]) / (nv - 1)
    _displace(o, moves, dxm, dvm)
    o.compute_map()
    return o.diagnostics()["emap"]


def test_emap_of_one_displaced_element_is_its_displacement():
    """Sites owned by the displaced element's neighbours next to it fall in
    the alpha range towards it, so the pair is compared; every other pair
    agrees.  E_map = |delta| in element spacings (Euclidean): the max norm
    would give 0.1, grid units four times the value."""
    e = _emap_of({(9, 9): (0.1, 0.05)})
    assert e == pytest.approx(math.hypot(0.1, 0.05), rel=1e-12)


def test_emap_uses_element_units_on_each_axis():
    """On a box whose element spacings differ between the axes (dx_m = 1/4,
    dv_m = 1/8) a displacement of 0.2 element spacings along v is 0.2, not
    0.2 * dv_m / dx_m or its square."""
    box = (-2.0, 2.0, -1.0, 1.0)
    e = _emap_of({(9, 9): (0.0, 0.2)}, box=box)
    assert e == pytest.approx(0.2, rel=1e-12)
    e2 = _emap_of({(9, 9): (0.2, 0.0)}, box=box)
    assert e2 == pytest.approx(0.2, rel=1e-12)


def test_emap_takes_the_largest_pair_mismatch():
    """Two displaced elements far apart: the larger displacement wins."""
    e = _emap_of({(5, 5): (0.05, 0.0), (13, 13): (-0.12, 0.09)})
    assert e == pytest.approx(math.hypot(0.12, 0.09), rel=1e-12)


# ---------------------------------------------------------------------------
# continuity of Q_r where Q(P, owner) jumps
# ---------------------------------------------------------------------------

def _curved_elements(o, eps):
    """Elements of the nonlinear map P = F(Q), x = q_x + eps sin(2 q_v) +
    eps q_x^2 / 2, v = q_v + eps sin(2 q_x): anchors F(Q_m), deformation
    T = dF/dQ and Hessian H = d2F/dQ2 at Q_m, so the second-order maps
    disagree between neighbours at third order in the element spacing."""
    el = o.elements()
    for m in range(o.ne):
        qx, qv = el[m, 0], el[m, 1]
        el[m] = [qx + eps * math.sin(2 * qv) + 0.5 * eps * qx * qx, qv + eps * math.sin(2 * qx),
                 1.0 + eps * qx, 2 * eps * math.cos(2 * qv), 2 * eps * math.cos(2 * qx), 1.0,
                 eps, 0.0, -4 * eps * math.sin(2 * qv),
                 -4 * eps * math.sin(2 * qx), 0.0, 0.0]
    o.set_elements(el)


def _boundary_jumps(o, eps):
    """Largest second difference across an ownership boundary along x, for
    Q_r and for the owner's own Q(P, m): Q(i+1) - Q(i) minus the mean of the
    one-sided steps on either side, which is O(dx^2) for a smooth map and
    O(jump) at a discontinuity."""
    _curved_elements(o, eps)
    _, qr = o.remap_resample()
    owner, _ = o.compute_map()
    tay = o.taylor()
    x = np.linspace(*BOX[:2], o.nx)
    v = np.linspace(*BOX[2:], o.nv)
    qo = np.empty((o.nx, o.nv))
    for i in range(o.nx):
        for j in range(o.nv):
            t = tay[owner[i, j]]
            qo[i, j] = t[12] + O.qofp(t, x[i], v[j])[0]
    jr = jo = 0.0
    for i in range(1, o.nx - 2):
        for j in range(o.nv):
            if owner[i, j] == owner[i + 1, j] or not (-1.0 < x[i] < 1.0 and -1.0 < v[j] < 1.0):
                continue
            for q, acc in ((qr[:, :, 0], "r"), (qo, "o")):
                d2 = (q[i + 1, j] - q[i, j]) - 0.5 * ((q[i, j] - q[i - 1, j]) + (q[i + 2, j] - q[i + 1, j]))
                if acc == "r":
                    jr = max(jr, abs(d2))
                else:
                    jo = max(jo, abs(d2))
    return jr, jo


@pytest.mark.parametrize("eps", [0.05, 0.15])
def test_blended_map_is_continuous_across_ownership_boundaries(eps):
    """eq. interpol: Q_r is continuous, the owner's map is not.  Halving the
    grid spacing at fixed element spacing (s = 4 -> 8) halves, at least, the
    second differences of Q_r across ownership boundaries, while those of
    Q(P, owner) keep the size of the mismatch between neighbours."""
    coarse = O.Oracle(65, 65, *BOX, 4, 0.01, 1000, 0.0)
    fine = O.Oracle(129, 129, *BOX, 8, 0.01, 1000, 0.0)
    for o in (coarse, fine):
        o.set_f(np.zeros((o.nx, o.nv)))
    jr_c, jo_c = _boundary_jumps(coarse, eps)
    jr_f, jo_f = _boundary_jumps(fine, eps)
    assert jo_f > 0.7 * jo_c          # the owner's map jumps: no shrinking
    assert jr_f < 0.5 * jr_c          # Q_r's second differences shrink
    assert jr_f < 0.2 * jo_f
