"""Host-side arithmetic of bench.py's roofline fields (no GPU)."""
import hashlib
import os

import pytest

import bench
from paper_1705_03750_gb300 import inputs as I


def test_step_bytes_per_update_matches_the_per_site_accounting():
    rc = I.HALOS_4096
    # FP32: f_ini 4 + f 4 + elements 304/64 + map 8 + remap 24/25
    assert bench.step_bytes_per_update(rc, True) == pytest.approx(4 + 4 + 4.75 + 8 + 0.96)
    assert bench.step_bytes_per_update(rc, False) == pytest.approx(8 + 8 + 4.75 + 8 + 0.96)


def test_map_algorithmic_bytes_are_one_slot_per_site_and_one_record_per_element():
    rc = I.HALOS_4096
    ne = 515 * 515
    b, units, _ = bench.algorithmic("claim_small", rc, True, ne)
    assert units == rc.nx * rc.nv and b == 4 * units + 128 * ne


def test_ncu_traffic_is_void_once_the_source_changed(monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1705_03750_gb300", "csrc", "map.cu")
    with open(src, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"claim_small": (123, "map.cu", sha[:16]),
                                               "reconstruct": (456, "map.cu", "0" * 16)})
    assert bench.ncu_traffic("claim_small") == 123
    assert bench.ncu_traffic("reconstruct") is None
    assert bench.ncu_traffic("spline_rows") is None
