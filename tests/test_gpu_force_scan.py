"""The GPU mass scan (Sec. 2.5, eq. of a(i)) against exact rational sums.

a(i) = 2 pi G [M_tot - M_left(i) - M_left(i-1)] is computed on the device
from the pixel masses M(i) with an error-free prefix (128-bit fixed point).
Here the GPU's own M(i) (read back) are summed exactly with Python
fractions; the GPU's a(i) must equal 2 pi G times the correctly rounded
exact bracket, up to one rounding of the product and the fixed-point
quantum of the masses (2^-112 of the largest), on grids whose row masses
span thirty orders of magnitude and both signs.  A plain FP64 scan misses
this by up to ~N ulps of M_tot where the bracket nearly cancels.
"""
import math
from fractions import Fraction

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


def _mixed_f(rc, seed, signed):
    rng = np.random.default_rng(seed)
    f = np.abs(rng.standard_normal((rc.nx, rc.nv)))
    scale = 10.0 ** (-(np.arange(rc.nx) * 7 % 31))
    if signed:
        scale *= np.where(rng.uniform(size=rc.nx) < 0.3, -1.0, 1.0)
    return f * scale[:, None]


def _check_exact(M, a, A):
    Mf = [Fraction(float(x)) for x in M]
    tot = sum(Mf)
    quantum = 2.0 ** -112 * float(np.abs(M).max()) * len(M) * A
    left_prev = Fraction(0)
    worst = 0.0
    for i, m in enumerate(Mf):
        left = left_prev + m
        ex = A * float(tot - left - left_prev)
        err = abs(a[i] - ex)
        bound = math.ulp(ex) + quantum
        assert err <= bound, f"i={i}: a={a[i]!r} exact={ex!r}"
        worst = max(worst, err / max(abs(A * float(tot)), 1e-300))
        left_prev = left
    return worst


@pytest.mark.parametrize("prec", [V.VM_FP64, V.VM_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("signed", [False, True], ids=["positive", "signed"])
def test_mass_scan_is_exact_on_mixed_magnitudes(prec, signed):
    rc = I.SPITZER_128.with_(nx=1531, nv=64)  # several pixels per thread, a ragged last chunk
    s = V.Solver(V.Config.from_run(rc, prec))
    s.set_f(_mixed_f(rc, 7, signed))
    s.reconstruct()
    df = s.density_force()
    _check_exact(df["M"], df["a"], 2 * math.pi * rc.G)


def test_mass_scan_of_a_cancelling_force():
    """The isothermal sheet is symmetric, so the bracket nearly cancels at
    the centre: there the exact result is tiny and the scan must still
    give it to its last bits."""
    rc = I.SPITZER_128.with_(nx=4097, nv=32)
    s = V.Solver(V.Config.from_run(rc))
    s.set_f(I.initial_f(rc))
    s.reconstruct()
    df = s.density_force()
    _check_exact(df["M"], df["a"], 2 * math.pi * rc.G)


def test_mass_scan_of_zero_mass():
    rc = I.SPITZER_128.with_(nx=64, nv=64)
    s = V.Solver(V.Config.from_run(rc))
    s.set_f(np.zeros((rc.nx, rc.nv)))
    s.reconstruct()
    df = s.density_force()
    assert not df["a"].any() and not df["da"].any() and not df["d2a"].any()
