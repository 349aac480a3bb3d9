"""The adaptive computing domain on the GPU (Sec. 2.2.1, eq. constrf; Sec.
2.3) against the oracle's: the existing lattice range and each map's site
rectangle identical, the influence map bit for bit on the same elements,
f within the reconstruction tolerance, through remaps (where the domain is
recomputed from the resampled f_ini)."""
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
# the apodised thermal-equilibrium sheet on a box about twice its support, remap every 10 steps
WIDE = I.APOD_128.with_(name="apod-wide", nx=192, nv=160, x_lo=-1.2, x_hi=1.2, v_lo=-1.6, v_hi=1.6, n_s=10)


def pair(rc, prec, f_th):
    cfg = V.Config.from_run(rc, PREC[prec])
    cfg.f_th = f_th
    s = V.Solver(cfg)
    o = O.Oracle(rc.nx, rc.nv, rc.x_lo, rc.x_hi, rc.v_lo, rc.v_hi, rc.s, rc.dt, rc.n_s, rc.G)
    o.set_fth(f_th)
    f0 = I.initial_f(rc)
    s.set_f(f0)
    o.set_f(f0)
    return s, o


def same_domain(s, o):
    d = s.diagnostics()
    od = o.domain()
    assert d["lattice_range"] == od["lattice"], (d["lattice_range"], od["lattice"])
    assert d["site_rect"] == od["rect"], (d["site_rect"], od["rect"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_domain_map_and_f_match_oracle_through_remaps(prec):
    s, o = pair(WIDE, prec, 1e-3)
    fi = o.fini()
    if prec == "fp32":
        fi = fi.astype(np.float32).astype(np.float64)        # the FP32 storage of the same cut f_ini
    assert np.array_equal(s.read_fini(), fi)
    for n in (1, 9, 1, 11):                                # remaps after steps 10 and 20
        s.step(n)
        o.step(n)
        fo = o.last_f()
        err = np.abs(s.read_f() - fo).max() / np.abs(fo).max()
        tol = 1e-6 if (prec == "fp64" or o.step_count <= 10) else 1e-5
        assert err <= tol, (o.step_count, err)
        # the map of the current elements, on both sides (the FP32 path's
        # elements follow its own force, so only the FP64 path has the
        # oracle's elements to the last bit)
        if prec == "fp64":
            s.compute_map()
            mo, _ = o.compute_map()
            same_domain(s, o)
            assert np.array_equal(s.read_map(), mo), o.step_count
        else:
            assert s.diagnostics()["lattice_range"] == o.domain()["lattice"]
    i0, i1, j0, j1 = s.diagnostics()["site_rect"]
    assert (i1 - i0 + 1) * (j1 - j0 + 1) < 0.4 * WIDE.nx * WIDE.nv   # a fraction of the box is worked


def test_full_domain_is_the_fixed_box_bit_for_bit():
    """An initial condition above f_th everywhere: every element exists, the
    rectangle is the grid, and the run is the fixed-box run bit for bit."""
    rc = I.SPITZER_128.with_(ic="blob", ic_params={"sx": 3.0, "sv": 5.0}, n_s=8)
    a = V.Solver(V.Config.from_run(rc, V.VM_FP32_MIXED))
    cfg = V.Config.from_run(rc, V.VM_FP32_MIXED)
    cfg.f_th = 1e-3
    b = V.Solver(cfg)
    f0 = I.initial_f(rc)
    a.set_f(f0)
    b.set_f(f0)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.read_f(), b.read_f())
    assert np.array_equal(a.elements(), b.elements())
    assert b.diagnostics()["lattice_range"] == (0, b.Lx - 1, 0, b.Lv - 1)


def test_nothing_above_the_threshold_gives_no_element_and_zero_f():
    s, o = pair(WIDE, "fp64", 10.0)
    s.step(12)
    o.step(12)
    assert not s.read_f().any()
    d = s.diagnostics()
    assert d["lattice_range"][1] < d["lattice_range"][0] and d["mass"] == 0.0


def test_checkpoint_keeps_the_domain(tmp_path):
    s, _ = pair(WIDE, "fp32", 1e-3)
    s.step(12)
    path = tmp_path / "dom.vlm"
    s.save(path)
    cfg = V.Config.from_run(WIDE, V.VM_FP32_MIXED)
    cfg.f_th = 1e-3
    t = V.Solver(cfg)
    t.load(path)
    assert t.diagnostics()["lattice_range"] == s.diagnostics()["lattice_range"]
    s.step(9)
    t.step(9)
    assert np.array_equal(s.read_f(), t.read_f())


def test_batch_refuses_the_adaptive_domain():
    cfg = V.Config.from_run(WIDE, V.VM_FP32_MIXED)
    cfg.f_th = 1e-3
    s = V.Solver(cfg)
    s.set_f(I.initial_f(WIDE))
    with pytest.raises(V.VlametError) as e:
        V.Batch([s], nstreams=1)
    assert e.value.status == 1
