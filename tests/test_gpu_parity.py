"""GPU (CUDA path through the C ABI) against the FP64 oracle.

Tolerances, per result (see the design notes for their derivation):
  * influence map: bit-exact (integer result of FP64 decisions taken in the
    same order on both sides), given identical element states;
  * f: |f_gpu - f_oracle| <= 1e-6 max|f| for both precisions;
  * pixel masses / total mass: FP64 path 1e-12 relative; FP32 path: the
    GPU's FP64 sum of its own FP32 f matches an exact sum of that f to 1e-12,
    and its deviation from the oracle's mass is bounded by the f tolerance;
  * elements after a step: FP64 path 1e-12 relative (the force differs only
    by summation order), FP32 path 1e-9 relative.
"""
import math

import numpy as np
import pytest

import oracle.oracle as O
from paper_1705_03750_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1705_03750_gb300 import build as B  # noqa: E402

B.build()
from paper_1705_03750_gb300 import vlamet as V  # noqa: E402

PREC = {"fp64": V.VM_FP64, "fp32": V.VM_FP32_MIXED}
F_TOL = 1e-6


def make(rc, prec="fp64", **kw):
    cfg = V.Config.from_run(rc, PREC[prec])
    for k, v in kw.items():
        setattr(cfg, k, v)
    s = V.Solver(cfg)
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G,
                 max_hole_rounds=kw.get("max_hole_rounds", 0))
    return s, o


def evolved_state(rc, steps):
    """Oracle elements after `steps` steps with no remap in between."""
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, 10 ** 6, rc.G)
    o.set_f(I.initial_f(rc))
    o.step(steps)
    return o.elements(), o.fini()


ELEMENT_TOL = {"fp64": (1e-13, 1e-12, 1e-10), "fp32": (1e-8, 1e-6, 1e-4)}


def element_errors(eg, eo):
    """Per state column, max |difference| over elements / max |value|."""
    scale = np.maximum(np.abs(eo).max(axis=0), 1e-300)
    return np.abs(eg - eo).max(axis=0) / scale


def assert_f_close(fg, fo, tol=F_TOL):
    scale = max(np.abs(fo).max(), 1e-300)
    err = np.abs(fg - fo).max() / scale
    assert err <= tol, f"max |df|/max|f| = {err:.3e}"
    return err


# ---------------------------------------------------------------------------
# the influence map: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("steps", [0, 19, 40, 150])
def test_map_bit_exact_on_injected_elements(prec, steps):
    rc = I.SPITZER_128
    s, o = make(rc, prec)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    if steps:
        el, _ = evolved_state(rc, steps)
        o.set_elements(el)
        s.set_elements(np.ascontiguousarray(el.T))
    s.compute_map()
    s.sync()
    mo, st = o.compute_map()
    assert st == 0
    mg = s.read_map()
    assert (mg == mo).all(), f"{(mg != mo).sum()} sites differ"
    d = s.diagnostics()
    stats = o.map_stats()
    assert d["holes"] == stats["holes"]
    if steps == 150:
        assert d["overflow_elements"] > 0      # the large-window path ran


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("steps", [40, 150])
def test_map_bit_exact_with_the_whole_lattice_window_alone(prec, steps):
    """Components leaving the 32 x 64 window go straight to the last tier
    (whole padded lattice, masks in global memory)."""
    rc = I.SPITZER_128
    s, o = make(rc, prec, map_windows=1)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    el, _ = evolved_state(rc, steps)
    o.set_elements(el)
    s.set_elements(np.ascontiguousarray(el.T))
    for _ in range(2):          # the second map reuses the cleared masks
        s.compute_map()
        s.sync()
        mo, st = o.compute_map()
        assert st == 0
        mg = s.read_map()
        assert (mg == mo).all(), f"{(mg != mo).sum()} sites differ"
    d = s.diagnostics()
    if steps == 150:
        assert d["overflow_elements"] > 0 and d["last_tier_elements"] == d["overflow_elements"]


@pytest.mark.parametrize("shape,s_", [((67, 45), 4), ((33, 33), 4), ((4, 4), 1), ((100, 37), 3)])
def test_map_ragged_and_tie_shapes(shape, s_):
    nx, nv = shape
    rc = I.SPITZER_128.with_(nx=nx, nv=nv, s=s_)
    if shape == (33, 33):       # exact ties: dx = dv = 1
        rc = rc.with_(x_lo=-16.0, x_hi=16.0, v_lo=-16.0, v_hi=16.0, G=0.0)
    s, o = make(rc)
    f0 = np.zeros((nx, nv)) if shape == (33, 33) else I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    for _ in range(2):
        s.step(3)
        o.step(3)
        s.compute_map()
        s.sync()
        mo, _ = o.compute_map()
        # oracle and GPU elements differ only by the force's summation order;
        # inject the oracle's to compare the decisions bit for bit
        s.set_elements(np.ascontiguousarray(o.elements().T))
        s.compute_map()
        assert (s.read_map() == mo).all()


def test_hole_repair_round_cap_reports_not_converged():
    rc = I.SPITZER_128.with_(nx=32, nv=32, s=2, dt=0.01)
    el, _ = evolved_state(rc, 80)          # needs several repair rounds
    s, o = make(rc, max_hole_rounds=1)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    o.set_elements(el)
    s.set_elements(np.ascontiguousarray(el.T))
    _, st = o.compute_map()
    assert st == 4
    s.compute_map()
    with pytest.raises(V.VlametError) as e:
        s.sync()
    assert e.value.status == 4
    s.sync()                                   # the error word was cleared


# ---------------------------------------------------------------------------
# reconstruction, masses and force on identical states
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("steps", [5, 19])
def test_reconstruct_and_force_on_injected_state(prec, steps):
    rc = I.SPITZER_128
    s, o = make(rc, prec)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    el, _ = evolved_state(rc, steps)
    o.set_elements(el)
    s.set_elements(np.ascontiguousarray(el.T))
    s.reconstruct()
    fo = o.reconstruct()
    fg = s.read_f()
    assert_f_close(fg, fo)
    dg, do = s.density_force(), o.density_force()
    Mt = do["Mtot"]
    if prec == "fp64":
        np.testing.assert_allclose(dg["M"], do["M"], rtol=0, atol=1e-12 * Mt)
        A = 2 * math.pi * rc.G * Mt
        np.testing.assert_allclose(dg["a"], do["a"], rtol=0, atol=1e-12 * A)
        np.testing.assert_allclose(dg["da"], do["da"], rtol=0, atol=1e-10 * np.abs(do["da"]).max())
        np.testing.assert_allclose(dg["d2a"], do["d2a"], rtol=0, atol=1e-8 * np.abs(do["d2a"]).max())
    else:
        f32 = s.read_f(dtype=np.float32)
        exact = np.array([math.fsum(r) for r in f32.astype(np.float64)]) * (rc.dx * rc.dv)
        np.testing.assert_allclose(dg["M"], exact, rtol=0, atol=1e-12 * Mt)
        np.testing.assert_allclose(dg["M"], do["M"], rtol=0, atol=F_TOL * np.abs(fo).max() * rc.nv * rc.dx * rc.dv)


# ---------------------------------------------------------------------------
# whole steps from the same initial condition
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_first_step_matches(prec):
    rc = I.SPITZER_128
    s, o = make(rc, prec)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    s.step(1)
    o.step(1)
    assert_f_close(s.read_f(), o.last_f())
    eg, eo = s.elements().T, o.elements()
    err = element_errors(eg, eo)
    # columns: x, v | T (4) | H (6); the force enters v at O(dt a), T through
    # a' and H through a'' (a second difference of the mass scan)
    lim = ELEMENT_TOL[prec]
    for c, e in enumerate(err):
        assert e <= lim[0 if c < 2 else (1 if c < 6 else 2)], (c, err)


@pytest.mark.parametrize("rc", [I.SPITZER_128, I.FREE_128], ids=["spitzer", "free"])
def test_fp64_path_tracks_oracle_over_200_steps(rc):
    s, o = make(rc)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    worst = 0.0
    for k in range(10):
        s.step(20)
        o.step(20)
        # after a remap: new f_ini and coefficients
        assert_f_close(s.read_fini(), o.fini())
        np.testing.assert_allclose(s.read_eta(), o.eta(), rtol=0, atol=1e-9 * np.abs(o.eta()).max())
        worst = max(worst, assert_f_close(s.read_f(), o.last_f()))
        dg, do = s.diagnostics(), o.diagnostics()
        assert dg["mass"] == pytest.approx(do["mass"], rel=1e-12, abs=1e-14)
        assert dg["energy"] == pytest.approx(do["energy"], rel=1e-10, abs=1e-12)
    assert worst < 1e-9


def test_fp32_path_error_against_oracle_over_100_steps():
    rc = I.SPITZER_128
    s, o = make(rc, "fp32")
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    errs = []
    for k in range(5):
        s.step(20)
        o.step(20)
        errs.append(np.abs(s.read_f() - o.last_f()).max() / np.abs(o.last_f()).max())
    # FP32 storage: each remap adds ~1e-7 relative rounding; the trajectories
    # then separate slowly (the system is not chaotic on this time scale)
    assert max(errs) < 1e-5, errs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_remap_on_injected_state(prec):
    rc = I.SPITZER_128
    el, fini = evolved_state(rc, 19)
    s, o = make(rc, prec)
    s.set_f(fini)
    o.set_f(fini)
    o.set_elements(el)
    s.set_elements(np.ascontiguousarray(el.T))
    fo, _ = o.remap_resample()
    s.remap()
    s.sync()
    assert_f_close(s.read_fini(), fo)


def test_zero_initial_condition():
    rc = I.SPITZER_128.with_(nx=48, nv=40)
    s, o = make(rc)
    s.set_f(np.zeros((48, 40)))
    s.step(25)
    assert (s.read_f() == 0).all() and (s.read_fini() == 0).all()
    d = s.density_force()
    assert (d["a"] == 0).all()


# ---------------------------------------------------------------------------
# the 4096^2 halo workload, one step and one remap, against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_halos_4096_first_step_full_grid(prec):
    rc = I.HALOS_4096
    s, o = make(rc, prec)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    s.step(1)
    o.step(1)
    assert_f_close(s.read_f(), o.last_f())
    dg, do = s.density_force(), o.density_force()
    tol = 1e-12 if prec == "fp64" else F_TOL * rc.nv * np.abs(o.last_f()).max() * rc.dx * rc.dv
    np.testing.assert_allclose(dg["M"], do["M"], rtol=0, atol=tol)
    s.compute_map()
    mo, _ = o.compute_map()
    s.set_elements(np.ascontiguousarray(o.elements().T))
    s.compute_map()
    assert (s.read_map() == mo).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("windows", [0, 1])
def test_halos_4096_evolved_state_transport_and_remap_full_grid(prec, windows):
    """The state the timed steps run on: 24 steps of the 4096^2 halo workload
    on the GPU (sheared elements, long boundary bands in the large map
    windows, certified FP32 decisions on the FP32-mixed path).  Its elements
    and its f_ini (widened from the stored precision) are injected into the
    oracle; then, on the full grid: one transport reconstruction (map bit for
    bit, f and M to the per-step bar), the remap (resampled f_ini and the
    spline coefficients of the row and column sweeps), and the first
    transport step after it (the step whose every Q_v lies on a node)."""
    rc = I.HALOS_4096
    cfg = V.Config.from_run(rc.with_(n_s=10 ** 6), PREC[prec])
    cfg.map_windows = windows
    s = V.Solver(cfg)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    s.step(rc.n_s - 1)
    s.sync()
    el = s.elements()
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, 10 ** 6, rc.G)
    o.set_f(s.read_fini())
    o.set_elements(np.ascontiguousarray(el.T))
    # transport reconstruction at the evolved elements
    s.reconstruct()
    fo = o.reconstruct()
    mo, _ = o.compute_map()
    assert (s.read_map() == mo).all()
    assert_f_close(s.read_f(), fo)
    dg, do = s.density_force(), o.density_force()
    tol = 1e-12 * do["Mtot"] if prec == "fp64" else F_TOL * rc.nv * np.abs(fo).max() * rc.dx * rc.dv
    np.testing.assert_allclose(dg["M"], do["M"], rtol=0, atol=tol)
    # the remap: Q_r blend, spline of f_ini, the new f_ini and its coefficients
    s.remap()
    o.remap()
    s.sync()
    fio = o.fini()
    assert_f_close(s.read_fini(), fio)
    # the spline system (rows (1, 4, 1)/6, diagonally dominant) has an
    # inverse of infinity-norm at most 1/(4/6 - 2/6) = 3 per axis, so an
    # error e of f_ini moves eta by at most 9 |e| (here e <= 1e-6 max f_ini),
    # plus the sweeps' own rounding (FP32: a few units of 6e-8 of max |eta|)
    eo = o.eta()
    if prec == "fp64":
        tol = 1e-12 * np.abs(eo).max()
    else:
        tol = 9 * F_TOL * np.abs(fio).max() + 1e-6 * np.abs(eo).max()
    assert np.abs(s.read_eta() - eo).max() <= tol
    # the first step after the remap, from each side's own state
    s.step(1)
    o.step(1)
    assert_f_close(s.read_f(), o.last_f())


# ---------------------------------------------------------------------------
# 8192^2: boundary components longer than every shared-memory window
# ---------------------------------------------------------------------------

def test_halos_8192_map_after_a_cycle_full_grid():
    rc = I.HALOS_8192
    s = V.Solver(V.Config.from_run(rc.with_(n_s=10 ** 6), V.VM_FP32_MIXED))
    f0 = I.initial_f(rc)
    s.set_f(f0)
    s.step(rc.n_s - 1)
    s.sync()
    el = s.elements()
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_f(f0)
    o.set_elements(np.ascontiguousarray(el.T))
    s.compute_map()
    s.sync()
    d = s.diagnostics()
    mo, st = o.compute_map()
    assert st == 0
    mg = s.read_map()
    assert (mg == mo).all(), f"{(mg != mo).sum()} sites differ"
    assert d["overflow_elements"] > 0


# ---------------------------------------------------------------------------
# the FP32-mixed reconstruction in tiles staged by bulk copies (recon_mode 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(4096, 4096), (130, 254), (97, 301), (64, 64)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_staged_tiles_match_oracle_and_the_row_kernel(shape):
    """Tiles of 4 x rows by 256 v columns, their f_ini patch staged in shared
    memory by bulk copies where it fits (nv % 4 == 0), global gathers where
    not (nv = 301, odd rows): one reconstruction of an evolved state against
    the oracle (f to the per-step bar, map bit for bit) and against the
    one-block-per-row kernel (f to rounding)."""
    nx, nv = shape
    rc = I.HALOS_4096.with_(nx=nx, nv=nv, s=8 if nx >= 1024 else 4)
    steps = 24 if nx >= 1024 else 18
    base = V.Config.from_run(rc.with_(n_s=10 ** 6), V.VM_FP32_MIXED)
    tiles = V.Config.from_run(rc.with_(n_s=10 ** 6), V.VM_FP32_MIXED)
    tiles.recon_mode = 1
    a, b = V.Solver(base), V.Solver(tiles)
    f0 = I.initial_f(rc)
    for s in (a, b):
        s.set_f(f0)
    b.step(steps)
    b.sync()
    el = b.elements()
    a.set_elements(np.ascontiguousarray(el))
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, 10 ** 6, rc.G)
    o.set_f(b.read_fini())
    o.set_elements(np.ascontiguousarray(el.T))
    b.reconstruct()
    a.reconstruct()
    fo = o.reconstruct()
    assert (b.read_map() == o.compute_map()[0]).all()
    fb = b.read_f()
    assert_f_close(fb, fo)
    assert np.abs(fb - a.read_f()).max() <= 1e-6 * np.abs(fo).max()
    db, do = b.density_force(), o.density_force()
    np.testing.assert_allclose(db["M"], do["M"], rtol=0, atol=F_TOL * rc.nv * np.abs(fo).max() * rc.dx * rc.dv)
    assert b.diagnostics()["bad_where"] == 0
