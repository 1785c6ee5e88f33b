"""CPU checks of bench.py's host-side pieces that its JSON line depends on:
the nvidia-smi clock summary (median under load, throttle reasons), recall@10,
the measured-peak lookup, and the rule that the committed DRAM-traffic
capture is reported only for the scan source, workload and nprobe it was
taken on."""
import json
import os

import numpy as np
import pytest

import bench


def _clocks(lines):
    c = bench.Clocks(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_median_under_load_and_reasons():
    idle = "345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = ["1995, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
            "2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2025, 2070, 940.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _clocks([idle] + busy + ["garbage line", "1, 2"])
    assert s["sm_mhz"] == 2025.0                      # idle sample below half the max left out
    assert s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    hot = _clocks(["1500, 2070, 1300.0, 0x8, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _clocks([]) is None and _clocks(["not, numbers, at, all, x, y, z, w"]) is None


def test_recall10_counts_set_overlap_of_the_first_ten():
    gt = np.arange(20).reshape(2, 10)
    ids = np.array([list(range(10)) + [99] * 5,          # all ten, extra columns ignored
                    [19, 18, 17, 16, 15, -1, -1, -1, -1, -1] + [10] * 5])
    assert bench.recall10(ids, gt) == pytest.approx((10 + 5) / 20)


def test_peaks_reads_the_measured_copy_bandwidth():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    bw, kind = bench.peaks()
    if os.path.exists(path):
        with open(path) as f:
            assert (bw, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert kind == "fallback"


def test_scan_traffic_only_for_its_own_source_workload_and_nprobe():
    t = bench.scan_traffic()
    if t is None:
        pytest.skip("the committed capture predates the current scan source")
    assert t["dram_bytes_per_search"] > 0 and t["dims_per_search"] > 0
    assert bench.scan_traffic(t["workload"], t["nprobe"]) is not None
    assert bench.scan_traffic(t["workload"], t["nprobe"] + 1) is None
    assert bench.scan_traffic("another_workload", t["nprobe"]) is None
    assert bench.scan_traffic(t["workload"], t["nprobe"], storage="bf16") is None
