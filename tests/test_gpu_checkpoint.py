"""Checkpoints through the C ABI (vm_save / vm_load): a solve resumed from a
checkpoint takes bit for bit the steps the saved solve takes, across a remap;
a checkpoint of another run is refused; an unreadable or foreign file is an
I/O error.  No oracle is involved: the property is exact self-consistency of
the state carried between steps (Sec. 2.4: elements; Secs. 2.2.2, 2.3.2:
f_ini and the spline coefficients; the position in the remap cycle)."""
import numpy as np
import pytest

from paper_1705_03750_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1705_03750_gb300 import build as B  # noqa: E402

B.build()
from paper_1705_03750_gb300 import vlamet as V  # noqa: E402

PREC = {"fp64": V.VM_FP64, "fp32": V.VM_FP32_MIXED}


def solver(rc, prec):
    return V.Solver(V.Config.from_run(rc, PREC[prec]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_is_bit_exact_across_a_remap(tmp_path, prec):
    # 128^2 halos, remap every 4 steps: 6 steps, save, then 7 more (two
    # remaps after the checkpoint, the first one step after it)
    rc = I.HALOS_4096.with_(nx=128, nv=128, s=4, n_s=4)
    a = solver(rc, prec)
    a.set_f(I.initial_f(rc))
    a.step(6)
    path = tmp_path / "state.vlm"
    a.save(path)
    a.step(7)
    f_a, el_a, fi_a = a.read_f(), a.elements(), a.read_fini()
    b = solver(rc, prec)
    b.load(path)
    b.step(7)
    f_b, el_b, fi_b = b.read_f(), b.elements(), b.read_fini()
    assert np.array_equal(el_a, el_b)
    assert np.array_equal(fi_a, fi_b)
    assert np.array_equal(f_a, f_b)
    assert np.array_equal(a.read_map(), b.read_map())


def test_resume_keeps_a_device_kept_cycle(tmp_path):
    # emap_remap > 0: the cycle and the forced-remap count live on the
    # device; a checkpoint carries them, and the resumed solve decides its
    # remaps (cycle end or E_map) as the saved one does
    rc = I.HALOS_4096.with_(nx=128, nv=128, s=4, n_s=5)
    f0 = I.initial_f(rc)

    def mk():
        cfg = V.Config.from_run(rc, PREC["fp32"])
        cfg.emap_remap = 1e-3           # small: some steps remap on E_map
        return V.Solver(cfg)

    a = mk()
    a.set_f(f0)
    a.step(7)
    path = tmp_path / "state.vlm"
    a.save(path)
    da = a.diagnostics()
    a.step(9)
    b = mk()
    b.load(path)
    db = b.diagnostics()
    assert (db["cycle"], db["emap_remaps"], db["step"]) == (da["cycle"], da["emap_remaps"], da["step"])
    b.step(9)
    assert a.diagnostics()["emap_remaps"] == b.diagnostics()["emap_remaps"]
    assert a.diagnostics()["cycle"] == b.diagnostics()["cycle"]
    assert np.array_equal(a.elements(), b.elements())
    assert np.array_equal(a.read_f(), b.read_f())


def test_load_refuses_another_run_and_bad_files(tmp_path):
    rc = I.HALOS_4096.with_(nx=128, nv=128, s=4, n_s=4)
    a = solver(rc, "fp64")
    with pytest.raises(V.VlametError) as e:
        a.save(tmp_path / "early.vlm")  # before set_f
    assert e.value.status == 7
    a.set_f(I.initial_f(rc))
    a.step(2)
    path = tmp_path / "state.vlm"
    a.save(path)
    for other in (rc.with_(nx=96), rc.with_(dt=rc.dt * 2)):
        with pytest.raises(V.VlametError) as e:
            solver(other, "fp64").load(path)
        assert e.value.status == 1
    with pytest.raises(V.VlametError) as e:
        solver(rc, "fp32").load(path)  # other precision
    assert e.value.status == 1
    junk = tmp_path / "junk.vlm"
    junk.write_bytes(b"not a checkpoint" * 8)
    for bad in (junk, tmp_path / "missing.vlm"):
        with pytest.raises(V.VlametError) as e:
            solver(rc, "fp64").load(bad)
        assert e.value.status == 9
    # a truncated checkpoint
    cut = tmp_path / "cut.vlm"
    cut.write_bytes(path.read_bytes()[:1000])
    with pytest.raises(V.VlametError) as e:
        solver(rc, "fp64").load(cut)
    assert e.value.status == 9


def test_resume_keeps_time_under_a_variable_time_step(tmp_path):
    """With C_dyn > 0 (Sec. 2.4) each step's dt comes from the density of the
    last f; the checkpoint carries the elapsed time and the last step, so
    after a resume vm_diag.time is still the sum of every step since
    vm_set_f and the steps that follow are the saved solve's."""
    rc = I.SPITZER_128.with_(n_s=4)
    cfg = V.Config.from_run(rc)
    cfg.c_dyn = 0.004
    a = V.Solver(cfg)
    a.set_f(I.initial_f(rc))
    a.step(6)
    t6 = a.diagnostics()["time"]
    path = tmp_path / "cdyn.vlm"
    a.save(path)
    b = V.Solver(cfg)
    b.load(path)
    db = b.diagnostics()
    assert db["time"] == t6 and db["last_dt"] == a.diagnostics()["last_dt"]
    a.step(7)
    b.step(7)
    da, db = a.diagnostics(), b.diagnostics()
    assert da["time"] == db["time"] and da["last_dt"] == db["last_dt"]
    assert 0.0 < da["last_dt"] < rc.dt
    assert np.array_equal(a.read_f(), b.read_f())
