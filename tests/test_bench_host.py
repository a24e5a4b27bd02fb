"""Host-side reporting logic of bench.py (CPU only): clock-sample parsing, the kernel name the
roofline reports, the step's launch form and the backward's byte count, and the rule that a stored DRAM-traffic figure is used only while the kernel
sources it was measured on are unchanged."""
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
    assert bench.spmm_kernel(256, 2) == "k_spmm_g4"          # BF16 512-byte rows: TMA gather4
    assert bench.spmm_kernel(256, 4) == "k_spmm_lring"       # 1 KB rows
    assert bench.spmm_kernel(16, 4) == "k_spmm"


def test_step_kernel_and_backward_bytes():
    # shiro_pack_spmm is one launch for FP32 rows of 512 bytes; BF16 rows of 512 bytes take the
    # pack and then the gather4 ring.
    assert bench.fused_step(128, 4) and not bench.fused_step(256, 2)
    assert not bench.fused_step(64, 4) and not bench.fused_step(256, 4)
    # The one-launch backward counts the pack of dC, the SpMM of A^T, one B row per non-empty row
    # of A^T and the dA values, each once (R-MAT 2^20 degree 16, N = 128, FP32: 2,970,272,864).
    K, nnz, RT, N, nzc = 1 << 20, 16086807, 1267409, 128, 547191
    assert bench.bwd_bytes(K, nnz, RT, N, 4, nzc) == 2970272864
    assert bench.bwd_bytes(K, nnz, RT, N, 4, nzc) == (bench.pack_bytes(RT, N, 4) +
                                                      bench.spmm_bytes(K, nnz, RT, N, 4) +
                                                      nzc * N * 4 + nnz * 4)


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    p = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(p))
    rec = {"kernel": "k_spmm_lean_dyn<float, float, 4, 1, 4, false>",
           "kernel_name": "k_spmm_lean_dyn", "workload": "rmat20_deg16_N128_4x4_f32",
           "sources_sha256": bench.sources_sha256(), "dram_bytes_per_launch": 123456}
    # A record taken on the current sources is used for its kernel and workload only ...
    p.write_text(json.dumps({"records": [rec]}))
    assert bench.traffic_from_profile("k_spmm_lean_dyn", "rmat20_deg16_N128_4x4_f32") == 123456
    assert bench.traffic_from_profile("k_spmm_lean_dyn", "rmat22_deg32_N256_4x4_bf16") is None
    assert bench.traffic_from_profile("k_sddmm_lean", "rmat20_deg16_N128_4x4_f32") is None
    # ... one taken on other sources is not, and neither is a missing record.
    p.write_text(json.dumps({"records": [dict(rec, sources_sha256="0" * 64)]}))
    assert bench.traffic_from_profile("k_spmm_lean_dyn", "rmat20_deg16_N128_4x4_f32") is None
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(tmp_path / "missing.json"))
    assert bench.traffic_from_profile("k_spmm_lean_dyn", "rmat20_deg16_N128_4x4_f32") is None


def test_traffic_record_from_ncu_csv(tmp_path, monkeypatch):
    """An ncu raw CSV export (a header row, a units row, one row per launch) becomes one record:
    the mean over the launches of the named kernel of DRAM bytes read + written."""
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(tmp_path / "traffic.json"))
    csv = tmp_path / "raw.csv"
    csv.write_text('"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum"\n'
                   '"","","Gbyte","Mbyte"\n'
                   '"0","k_pack_rows<float>","1.5","10"\n'
                   '"1","k_spmm_lean_dyn<float, float, 4, 1, 4, false>","1.0","500"\n'
                   '"2","k_spmm_lean_dyn<float, float, 4, 1, 4, false>","2.0","700"\n')
    bench.write_traffic_record(str(csv), "k_spmm_lean_dyn<float, float, 4, 1, 4, false>",
                               "rmat20_deg16_N128_4x4_f32", "ncu ...")
    r = json.load(open(tmp_path / "traffic.json"))["records"]
    assert len(r) == 1 and r[0]["launches"] == 2
    assert r[0]["dram_bytes_per_launch"] == int((1.0e9 + 0.5e9 + 2.0e9 + 0.7e9) / 2)
    assert bench.traffic_from_profile("k_spmm_lean_dyn", "rmat20_deg16_N128_4x4_f32") == r[0]["dram_bytes_per_launch"]


def test_l2_ceiling_fold_and_forms_parsing():
    a = bench.parse(["--forms", "gcn,er"])
    assert bench.forms_of(a) == {"gcn", "er"} and a.seed == 2
    assert bench.forms_of(bench.parse(["--no-forms"])) == set()
    assert bench.forms_of(bench.parse([])) == set(bench.FORMS)
    assert bench.parse(["--scale", "22", "--deg", "32"]).seed == 3
    # The algorithmic byte counts of the JSON line.
    assert bench.spmm_bytes(10, 20, 5, 4, 2) == 11 * 8 + 20 * 8 + 5 * 4 * 2 + 10 * 4 * 4
    assert bench.pack_bytes(5, 4, 2) == 2 * 5 * 4 * 2 + 5 * 4
    assert bench.sddmm_bytes(10, 20, 5, 4, 4) == 20 * 8 + 10 * 4 * 4 + 5 * 4 * 4 + 20 * 4


def test_traffic_record_from_metrics_log(tmp_path, monkeypatch):
    """The long form of ncu's --metrics --csv log (one row per launch and metric)."""
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(tmp_path / "traffic.json"))
    csv = tmp_path / "log.csv"
    csv.write_text('==PROF== Connected to process 1\n'
                   '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
                   '"0","void shiro::k_spmm_lean_fused<float>(P)","dram__bytes_read.sum","byte","3000"\n'
                   '"0","void shiro::k_spmm_lean_fused<float>(P)","dram__bytes_write.sum","byte","1000"\n'
                   '"0","void shiro::k_spmm_lean_fused<float>(P)","gpu__time_duration.sum","ns","5"\n'
                   '"1","void shiro::k_spmm_lean_fused<float>(P)","dram__bytes_read.sum","byte","5000"\n'
                   '"1","void shiro::k_spmm_lean_fused<float>(P)","dram__bytes_write.sum","byte","1000"\n')
    bench.write_traffic_record(str(csv), "k_spmm_lean_fused<float>", "w", "ncu ...")
    r = json.load(open(tmp_path / "traffic.json"))["records"][0]
    assert r["launches"] == 2 and r["dram_bytes_per_launch"] == 5000
