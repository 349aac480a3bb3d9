"""The C-ABI library loads and exports every entry point include/*.h declares;
host-only calls behave as documented.  No GPU needed (no compute calls)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_03750_gb300 import build as B
    B.build()
    from paper_1705_03750_gb300 import vlamet as V
    return V.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(vm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    from paper_1705_03750_gb300 import vlamet as V
    assert declared == set(V.EXPORTS), declared ^ set(V.EXPORTS)
    so = os.path.join(ROOT, "paper_1705_03750_gb300", "_lib", "libvlamet.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vm_[a-z0-9_]+)$", out, flags=re.M))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)


def test_host_only_calls(lib):
    from paper_1705_03750_gb300 import vlamet as V
    c = V.VmConfig()
    lib.vm_config_default(C.byref(c))
    assert c.alpha == pytest.approx(3 ** 0.5 / 4) and c.beta == pytest.approx(0.5 * (1 - 3 ** 0.5 / 2))
    assert lib.vm_workspace_bytes(C.byref(c)) == 0          # nx = nv = 0 is invalid
    cfg = V.Config(128, 128, -1, 1, -2.5, 2.5, 4, 0.005, 20, 1.0)
    n64 = V.workspace_bytes(cfg)
    cfg32 = V.Config(128, 128, -1, 1, -2.5, 2.5, 4, 0.005, 20, 1.0, precision=V.VM_FP32_MIXED)
    n32 = V.workspace_bytes(cfg32)
    assert n64 > n32 > 128 * 128 * 16
    bad = V.Config(3, 128, -1, 1, -2.5, 2.5, 4, 0.005, 20, 1.0)
    assert V.workspace_bytes(bad) == 0
    bad = V.Config(128, 128, 1, -1, -2.5, 2.5, 4, 0.005, 20, 1.0)
    assert V.workspace_bytes(bad) == 0
    assert lib.vm_status_string(5).decode().startswith("influence region")
    h = C.c_void_p()
    # a bad config is refused before any device work
    assert lib.vm_create(C.byref(bad.c()), C.c_void_p(256), 1 << 30, None, C.byref(h)) == 1
    assert lib.vm_create(C.byref(cfg.c()), C.c_void_p(256), 16, None, C.byref(h)) == 2
    assert lib.vm_create(C.byref(cfg.c()), C.c_void_p(257), n64, None, C.byref(h)) == 1


def test_solver_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1705_03750_gb300 import vlamet as V
    with pytest.raises(RuntimeError):
        V.Solver(V.Config(64, 64, -1, 1, -1, 1, 4, 0.01, 10, 1.0))


def test_product_path_does_not_import_the_oracle():
    for f in glob.glob(os.path.join(ROOT, "paper_1705_03750_gb300", "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
            assert "vlamet_oracle" not in txt and "oracle/" not in txt, f


def test_binding_refuses_arrays_the_call_would_read_past():
    """The C ABI takes bare pointers: the binding checks shape, dtype and
    layout first (a smaller buffer would be read past its end)."""
    import types

    import numpy as np

    from paper_1705_03750_gb300 import vlamet as V
    fake = types.SimpleNamespace(device=None)
    ok = np.zeros((8, 6))
    p, dev = V.Solver._arg(fake, ok, (8, 6), "float64")
    assert dev == 0 and p.value == ok.ctypes.data
    for bad in (np.zeros((6, 8)), np.zeros((8, 6), dtype=np.float32), np.zeros((8, 12))[:, ::2]):
        with pytest.raises(ValueError):
            V.Solver._arg(fake, bad, (8, 6), "float64")


def test_4d_host_only_calls(lib):
    import ctypes as C
    from paper_1705_03750_gb300 import inputs4d as I4
    from paper_1705_03750_gb300 import vlamet4d as V4
    good = V4.config(I4.HALOS4D_16)
    n = V4.workspace_bytes(good)
    assert n > 16 ** 4 * (3 * 8 + 16 + 4 * 4)
    bad = V4.config(I4.HALOS4D_16.with_(n=(3, 16, 16, 16)))
    assert V4.workspace_bytes(bad) == 0
    bad = V4.config(I4.HALOS4D_16.with_(s=9))
    assert V4.workspace_bytes(bad) == 0
    h = C.c_void_p()
    # refused before any device work: a bad config, a misaligned or short workspace
    assert lib.vm_4d_create(C.byref(bad), C.c_void_p(256), 1 << 30, None, C.byref(h)) == 1
    assert lib.vm_4d_create(C.byref(good), C.c_void_p(257), n, None, C.byref(h)) == 1
    assert lib.vm_4d_create(C.byref(good), C.c_void_p(256), 16, None, C.byref(h)) == 2
    assert lib.vm_4d_kernel_name(2).decode() == "percolate"
    assert lib.vm_4d_kernel_name(99) is None
