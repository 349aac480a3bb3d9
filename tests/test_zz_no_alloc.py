"""The allocation-free force entry point against the solver's own.

vm_force_from_f_static serves callers that cannot allocate device memory
(a host application that owns the device heap, or a loop that must not pay
for cudaMalloc/cudaFree synchronisation): its only scratch is a static
device array shared by all calls.  Two calls in a row, on different grids,
must each give what vm_reconstruct + vm_density_force give for the same f
(at initialisation the transport reconstruction returns f_ini exactly),
within the tolerances of the reconstruction parity test.  This file sorts
last so that a run stopping at the first failure has run everything else.
"""
import math

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


def _reference(rc):
    """M, a, a', a'' from the solver's entry points for f0 at t = 0."""
    s = V.Solver(V.Config.from_run(rc))
    f0 = I.initial_f(rc)
    s.set_f(f0)
    s.reconstruct()
    return f0, s.density_force()


def _static(rc, f0):
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.from_numpy(f0).to(dev)
    out = {k: torch.full((rc.nx,), float("nan"), dtype=torch.float64, device=dev) for k in ("M", "a", "da", "d2a")}
    V.force_from_f_static(f, V.Config.from_run(rc), out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _close(got, ref, rc):
    Mt = ref["M"].sum()
    np.testing.assert_allclose(got["M"], ref["M"], rtol=0, atol=1e-12 * Mt)
    A = 2 * math.pi * rc.G * Mt
    np.testing.assert_allclose(got["a"], ref["a"], rtol=0, atol=1e-12 * A)
    np.testing.assert_allclose(got["da"], ref["da"], rtol=0, atol=1e-10 * np.abs(ref["da"]).max())
    np.testing.assert_allclose(got["d2a"], ref["d2a"], rtol=0, atol=1e-8 * np.abs(ref["d2a"]).max())


def test_static_force_matches_solver_on_two_calls_in_a_row():
    rc1 = I.SPITZER_128
    rc2 = I.HALOS_4096.with_(nx=1000, nv=700)
    f1, ref1 = _reference(rc1)
    f2, ref2 = _reference(rc2)
    _close(_static(rc1, f1), ref1, rc1)     # first call (sets up the scratch address)
    _close(_static(rc2, f2), ref2, rc2)     # second call reuses the scratch, other size
    _close(_static(rc1, f1), ref1, rc1)     # and back: nothing left over from the larger grid


def test_static_force_refuses_grids_beyond_the_scratch():
    rc = I.SPITZER_128.with_(nx=V.VM_STATIC_FORCE_MAX_NX + 1, nv=4)
    with pytest.raises(ValueError, match="static scratch limit"):
        V.force_from_f_static(torch.zeros((rc.nx, rc.nv), dtype=torch.float64, device="cuda"),
                              V.Config.from_run(rc), {})
    # the C entry point itself refuses too, before touching the device
    import ctypes as C
    dev_buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dev_buf.data_ptr())
    st = V.load().vm_force_from_f_static(p, V.VM_DTYPE_F64, V.VM_STATIC_FORCE_MAX_NX + 1, 8, -1.0, 1.0, -1.0, 1.0,
                                         1.0, 0, None, p, p, p, None)
    assert st == 1
