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
    b, units, _ = bench.algorithmic("claim_pair", rc, True, ne)
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


def test_issue_roofline_counts_one_instruction_per_scheduler_per_clock(monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1705_03750_gb300", "csrc", "map.cu")
    with open(src, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    monkeypatch.setattr(bench, "NCU_INSTR", {"claim_pair": (1_000_000, "map.cu", sha[:16]),
                                             "reconstruct": (1_000_000, "map.cu", "0" * 16)})
    r = bench.issue_roofline("claim_pair", 1e-3, 2000.0)
    assert r["peak"] == pytest.approx(4 * 152 * 2000e6)
    assert r["achieved"] == pytest.approx(1e9)
    assert r["frac"] == pytest.approx(1e9 / (4 * 152 * 2000e6))
    assert bench.issue_roofline("reconstruct", 1e-3, 2000.0) is None  # source changed
    assert bench.issue_roofline("claim_pair", 1e-3, None) is None     # no clock sample


def test_prefix_key_hashes_the_source_before_the_marked_section(monkeypatch):
    # a key over the translation unit's text before a section stays valid when
    # only code after it changes, and is void when code before it changes
    src = os.path.join(bench.ROOT, "paper_1705_03750_gb300", "csrc", "phase4d.cu")
    with open(src, "rb") as fh:
        text = fh.read()
    marker = bench.PHASE4D_PREFIX_END
    i = text.index(marker.encode())
    prefix = text[:text.rindex(b"\n// ----", 0, i)]
    sha = hashlib.sha256(prefix).hexdigest()[:16]
    monkeypatch.setattr(bench, "NCU4_INSTR", {"percolate": (7, "phase4d.cu", sha),
                                              "other": (8, "phase4d.cu", "0" * 16)})
    assert bench._keyed(bench.NCU4_INSTR, "percolate", marker) == 7
    assert bench._keyed(bench.NCU4_INSTR, "other", marker) is None
    assert bench._keyed(bench.NCU4_INSTR, "percolate", "no such marker in the file") is None
    full = hashlib.sha256(text).hexdigest()[:16]
    assert full != sha and bench._keyed({"k": (9, "phase4d.cu", full)}, "k") == 9
