"""4D phase-space (2D space) CUDA path against the FP64 oracle, through the C ABI.

The influence map must be bit-exact for the same elements; f, f_ini and eta
are computed in the oracle's operation order and must agree to rounding
(1e-12 of max f; the bar is 1e-6); pixel masses and the field are summed in
another order (1e-12 relative); over several steps with remaps the element
trajectories carry that rounding along (f within 1e-9 of max f).
"""
import numpy as np
import pytest

import oracle.oracle4d as Q
from paper_1705_03750_gb300 import inputs4d as I4

pytestmark = pytest.mark.gpu


def _pair(rc):
    from paper_1705_03750_gb300 import vlamet4d as V4
    s = V4.Solver4D(V4.config(rc))
    o = Q.Oracle4D.from_run(rc)
    f0 = I4.initial_f4(rc)
    s.set_f(f0)
    o.set_f(f0)
    return s, o, f0


def _distort(o, rc, seed=7, amp=0.1, hamp=0.05, disp=0.2):
    el = o.elements()
    rng = np.random.default_rng(seed)
    dm = np.array(rc.d) * rc.s
    for m in range(o.ne):
        el[m, 4:20] = (np.eye(4) + amp * rng.normal(size=(4, 4))).ravel()
        el[m, 20:60] = hamp * rng.normal(size=40)
        el[m, 0:4] += disp * rng.normal(size=4) * dm
    return el


@pytest.mark.parametrize("name", ["halos4d-16^4", "halos4d-18x14x20x12"])
def test_spline_coefficients_match_oracle(name):
    rc = I4.WORKLOADS4D[name]
    s, o, f0 = _pair(rc)
    eta = s.read_eta()
    assert np.abs(eta - o.eta()).max() <= 1e-13 * np.abs(o.eta()).max()
    np.testing.assert_array_equal(s.read_fini(), f0)


@pytest.mark.parametrize("name", ["halos4d-16^4", "halos4d-18x14x20x12"])
def test_map_and_reconstruction_on_a_distorted_state(name):
    rc = I4.WORKLOADS4D[name]
    s, o, f0 = _pair(rc)
    el = _distort(o, rc)
    o.set_elements(el)
    s.set_elements(el)
    fo = o.reconstruct()
    s.reconstruct()
    s.sync()
    mo = o.last_map()
    st = o.map_stats()
    assert st["multi_claims"] > 0
    mg = s.read_map()
    assert (mg == mo).all(), int((mg != mo).sum())
    fg = s.read_f()
    assert np.abs(fg - fo).max() <= 1e-12 * np.abs(fo).max()
    do = o.density_force()
    dg = s.density_force()
    np.testing.assert_allclose(dg["M"], do["M"], rtol=1e-12, atol=1e-15 * np.abs(do["M"]).max())
    scale = np.abs(do["field"]).max(axis=(0, 1))
    assert (np.abs(dg["field"] - do["field"]).max(axis=(0, 1)) <= 1e-10 * scale).all()


def test_components_larger_than_the_window_are_filled_over_the_whole_lattice():
    # a strong second-order term stretches components far beyond the
    # shared-memory window; those elements take the whole-lattice pass
    rc = I4.HALOS4D_16.with_(n=(9, 8, 10, 9), s=3)
    s, o, f0 = _pair(rc)
    el = _distort(o, rc, amp=0.15, hamp=0.3, disp=0.2)
    o.set_elements(el)
    s.set_elements(el)
    fo = o.reconstruct()
    s.reconstruct()
    s.sync()
    assert s.map_stats()["window_overflows"] > 0
    assert (s.read_map() == o.last_map()).all()
    assert np.abs(s.read_f() - fo).max() <= 1e-12 * np.abs(fo).max()


@pytest.mark.parametrize("distort", [False, True])
def test_holes_are_repaired_like_the_oracle(distort):
    # a one-site connectivity margin keeps the outer elements from
    # percolating, leaving unexplored sites along the grid's edge
    from paper_1705_03750_gb300 import vlamet4d as V4
    rc = I4.HALOS4D_16.with_(n=(13, 11, 12, 10), s=4)
    s = V4.Solver4D(V4.config(rc, pad=1))
    o = Q.Oracle4D.from_run(rc, pad=1)
    f0 = I4.initial_f4(rc)
    s.set_f(f0)
    o.set_f(f0)
    if distort:
        el = _distort(o, rc, seed=5, amp=0.1, hamp=0.3, disp=0.1)
        o.set_elements(el)
        s.set_elements(el)
    fo = o.reconstruct()
    assert o.map_stats()["holes"] > 0
    s.reconstruct()
    s.sync()
    st = s.map_stats()
    assert st["holes"] == o.map_stats()["holes"] and st["rounds"] == o.map_stats()["rounds"]
    assert (s.read_map() == o.last_map()).all()
    assert np.abs(s.read_f() - fo).max() <= 1e-12 * np.abs(fo).max()


@pytest.mark.parametrize("name", ["halos4d-16^4", "halos4d-18x14x20x12"])
def test_remap_on_a_distorted_state_matches_oracle(name):
    rc = I4.WORKLOADS4D[name]
    s, o, f0 = _pair(rc)
    el = _distort(o, rc, amp=0.05, hamp=0.1, disp=0.1)
    o.set_elements(el)
    s.set_elements(el)
    o.remap()
    s.remap()
    s.sync()
    fo = o.fini()
    assert np.abs(s.read_fini() - fo).max() <= 1e-12 * np.abs(fo).max()
    eo = o.eta()
    assert np.abs(s.read_eta() - eo).max() <= 1e-12 * np.abs(eo).max()
    np.testing.assert_array_equal(s.elements(), o.elements())


@pytest.mark.parametrize("name", ["halos4d-16^4", "halos4d-18x14x20x12", "free4d-16^4-G0"])
def test_steps_through_two_remaps_match_oracle(name):
    rc = I4.WORKLOADS4D[name]
    s, o, f0 = _pair(rc)
    for k in range(rc.steps):              # n_s = 4: remaps after steps 4 and 8
        s.step(1)
        o.step(1)
        fg = s.read_f()
        fo = o.last_f()
        err = np.abs(fg - fo).max() / np.abs(fo).max()
        assert err <= 1e-9, (k, err)
    np.testing.assert_allclose(s.elements(), o.elements(), rtol=0, atol=1e-9)
    assert np.abs(s.read_fini() - o.fini()).max() <= 1e-9 * np.abs(o.fini()).max()


def test_full_size_map_and_reconstruction_after_a_cycle():
    # the measured workload (64^4, 16.8 M sites) after one remap cycle and
    # three more steps; the oracle rebuilds the map and f from the GPU's
    # elements and f_ini
    rc = I4.HALOS4D_64
    from paper_1705_03750_gb300 import vlamet4d as V4
    s = V4.Solver4D(V4.config(rc))
    f0 = I4.initial_f4(rc)
    s.set_f(f0)
    s.step(rc.n_s + 3)
    s.sync()
    el = s.elements()
    fini = s.read_fini()
    s.reconstruct()
    s.sync()
    o = Q.Oracle4D.from_run(rc)
    o.set_f(fini)
    o.set_elements(el)
    fo = o.reconstruct()
    assert (s.read_map() == o.last_map()).all()
    assert np.abs(s.read_f() - fo).max() <= 1e-12 * np.abs(fo).max()


def test_diagnostics_match_oracle():
    rc = I4.HALOS4D_16
    s, o, f0 = _pair(rc)
    for k in (0, 3):
        if k:
            s.step(k)
            o.step(k)
        dg = s.diagnostics()
        do = o.diagnostics()
        for key in ("mass", "ekin", "epot"):
            assert dg[key] == pytest.approx(do[key], rel=1e-10), (k, key)
        assert dg["detT_min"] == pytest.approx(do["detT_min"], abs=1e-12)
        assert dg["detT_max"] == pytest.approx(do["detT_max"], abs=1e-12)
