"""Host logic of bench.py's clock record (no GPU, no nvidia-smi): the summary
keeps the samples that arrived while the timed region ran, falls back to the
next sample for a region shorter than the sampling interval, and reports
every throttle reason seen; and the ncu counter table is void once the
kernel's source file no longer has the captured hash."""
import bench


def _line(sm, mx=2070, reasons=("Not Active",) * 4):
    # index, clocks.sm, clocks.max.sm, power.draw, active mask, then the four reasons
    return ", ".join(["0", str(sm), str(mx), "900.0", "0x0"] + list(reasons)) + "\n"


def _sampler(lines, t_begin, t_end):
    s = bench.ClockSampler("0")
    s.lines = lines
    s.t_begin, s.t_end = t_begin, t_end
    return s


def test_summary_keeps_only_the_samples_of_the_timed_region():
    lines = [(0.00, _line(1200)), (0.10, _line(2070)), (0.12, _line(2055)), (0.14, _line(2070)),
             (0.30, _line(900))]
    st = _sampler(lines, 0.09, 0.15).summary()
    assert st["samples"] == 3 and st["sm_mhz"] == 2070 and st["sm_max_mhz"] == 2070 and st["reasons"] == []


def test_a_region_shorter_than_the_interval_takes_the_next_sample():
    lines = [(0.00, _line(1500)), (0.50, _line(2070))]
    st = _sampler(lines, 0.10, 0.105).summary()
    assert st["samples"] == 1 and st["sm_mhz"] == 2070


def test_throttle_reasons_seen_during_the_region_are_reported():
    hot = ("Not Active", "Active", "Not Active", "Active")  # hw_slowdown .. sw_power_cap
    lines = [(0.00, _line(2070, reasons=("Active",) * 4)), (0.11, _line(1900, reasons=hot)), (0.12, _line(2070))]
    st = _sampler(lines, 0.10, 0.13).summary()
    assert st["samples"] == 2
    assert st["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_no_samples_is_reported_as_such():
    st = _sampler([], 0.0, 1.0).summary()
    assert st["sm_mhz"] is None and st["reasons"] == ["no samples"]


def test_ncu_counters_are_void_once_their_source_changed():
    assert bench._keyed({"k": (123, "map.cu", "0" * 16)}, "k") is None
    assert bench._keyed({}, "k") is None
    ent = bench.NCU_TRAFFIC["claim_pair"]
    assert bench._keyed({"k": ent}, "k") in (ent[0], None)
