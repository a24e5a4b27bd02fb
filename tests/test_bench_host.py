"""Host-side reporting logic of bench.py (CPU only): clock-sample parsing, the kernel name the
roofline reports, and the rule that a stored DRAM-traffic figure is used only while the kernel
sources it was measured on are unchanged."""
import hashlib
import json
import os

import bench


def _line(sm, mx, hw="Not Active", power="Not Active"):
    # timestamp, index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"2026/01/01 00:00:00.000, 0, {sm}, {mx}, 900.0, 0x0, {hw}, Not Active, Not Active, {power}"


def test_clock_summary_median_under_load_and_reasons():
    c = bench.ClockSampler(0)
    c.lines = [_line(345, 2070), _line(2070, 2070), _line(2070, 2070, power="Active"),
               _line(2055, 2070), _line(400, 2070)]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0          # idle edges (below half the maximum) dropped
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 5
    c.lines = [_line(1500, 2070, hw="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown"]
    c.lines = ["garbage"]
    assert c.summary()["sm_mhz"] is None


def test_spmm_kernel_names():
    assert bench.spmm_kernel(128, 4) == "k_spmm_lean_dyn"    # FP32 N = 128, 512-byte rows
    assert bench.spmm_kernel(32, 4) == "k_spmm_lean_dyn"     # 128-byte rows
    assert bench.spmm_kernel(128, 2) == "k_spmm_lean"        # BF16 256-byte rows: one item per warp
    assert bench.spmm_kernel(256, 2) == "k_spmm_lean_dyn"
    assert bench.spmm_kernel(256, 4) == "k_spmm_lring"       # 1 KB rows
    assert bench.spmm_kernel(16, 4) == "k_spmm"


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        h.update(open(os.path.join(bench.ROOT, f), "rb").read())
    p = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(p))
    # A record taken on the current sources is used ...
    p.write_text(json.dumps({"kernel_sources_sha256": h.hexdigest(),
                             "dram_bytes_per_launch": 123456}))
    assert bench.traffic_from_profile() == 123456
    # ... one taken on other sources is not, and neither is a missing record.
    p.write_text(json.dumps({"kernel_sources_sha256": "0" * 64, "dram_bytes_per_launch": 1}))
    assert bench.traffic_from_profile() is None
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(tmp_path / "missing.json"))
    assert bench.traffic_from_profile() is None
