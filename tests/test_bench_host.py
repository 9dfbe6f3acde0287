"""Host logic of bench.py's timing rules on CPU: the clock record taken
during a timed region (nvidia-smi samples), the rule that rejects a run, the
roofline denominator and the walk-traffic lookup key."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary_of(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(line + "\n" for line in lines))
    clk = bench.ClockSampler(0)
    clk.path = str(path)
    return clk.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    na, act = "Not Active", "Active"
    rows = [f"0, {mhz}, 2070, 900.5, 0x0, {na}, {na}, {na}, {cap}"
            for mhz, cap in ((2070, na), (1995, act), (2070, na), (2055, na), (1980, act))]
    s = _summary_of(tmp_path, ["garbage line", *rows])
    assert s["samples"] == 5
    assert s["sm_mhz"] == 2055.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert not bench.rejected(s)  # a power cap is kept and noted


def test_thermal_or_hardware_slowdown_rejects(tmp_path):
    na, act = "Not Active", "Active"
    for col in range(3):  # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown
        flags = [na, na, na, na]
        flags[col] = act
        s = _summary_of(tmp_path, [f"0, 1800, 2070, 1200.0, 0x0, {', '.join(flags)}"])
        assert bench.rejected(s), col


def test_clock_stuck_low_without_a_reason_rejects():
    assert bench.rejected({"sm_mhz": 900.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert not bench.rejected({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert not bench.rejected({"sm_mhz": 900.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]})


def test_missing_clock_record_is_reported_not_invented(tmp_path):
    s = _summary_of(tmp_path, [])
    assert s["samples"] == 0 and s["sm_mhz"] is None
    assert not bench.rejected(s)


def test_roofline_peak_comes_from_the_measured_file():
    value, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and value == float(json.load(open(path))["hbm_gbs"])
    else:
        assert kind == "fallback" and value == bench.FALLBACK_HBM_GBS


def test_walk_traffic_is_keyed_by_the_walk_sources():
    prof = json.load(open(bench.WALK_PROFILE))
    assert set(prof["dram_bytes_per_launch_by_seg_target"]) == {"8", "16", "32"}
    for t, (rd, wr) in prof["dram_read_write_by_seg_target"].items():
        assert prof["dram_bytes_per_launch_by_seg_target"][t] == rd + wr
    # the hash covers exactly the files the walk kernel is compiled from
    assert all(os.path.exists(os.path.join(ROOT, p)) for p in bench.WALK_SOURCES)
    assert len(bench.sources_hash()) == 16
