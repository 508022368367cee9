"""The arithmetic of bench.py's JSON line, on CPU: the HBM roofline from algorithmic bytes,
the compute-side rooflines (warp-instruction issue for FP32+refine against the device's SM
count, the FP64 pipe for FP64 against the measured FMA rate),
and the ncu table's gate on the kernel source (its figures only count while the profiled
source is unchanged).  No GPU."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_compute_roofline_fp64_counts_pipe_operations_against_the_measured_peak():
    fp64 = {"tflops": 1.0}  # 0.5e12 FMA per second
    r = bench.compute_roofline("f64", rows=67_108_864, ms_step=0.762, sm_mhz=2070.0, sms=152, fp64=fp64)
    assert r["bound"] == "fp64" and r["peak_kind"].startswith("measured")
    assert r["achieved"] == pytest.approx(5 * 67_108_864 / 0.762e-3)  # 4 FMA + 1 MUL a row
    assert r["peak"] == pytest.approx(0.5e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 0.5e12)
    assert r["tflops"] == pytest.approx(9 * 67_108_864 / 0.762e-3 / 1e12)
    assert bench.compute_roofline("f64", 1, 1.0, 2070.0, 152, None) is None  # no measured peak, no figure


def test_compute_roofline_issue_uses_the_table_the_sm_count_and_the_sampled_clock(monkeypatch):
    monkeypatch.setattr(bench, "profile_entry", lambda v: {"warp_inst_per_row": 8.0})
    r = bench.compute_roofline("f32_refine", rows=1_000_000, ms_step=0.5, sm_mhz=2000.0, sms=148)
    assert r["bound"] == "issue"
    assert r["achieved"] == pytest.approx(8.0 * 1e6 / 0.5e-3)
    assert r["peak"] == pytest.approx(148 * 4 * 2000.0e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.compute_roofline("f32_refine", 1, 1.0, None, 152) is None  # no clock sample, no figure
    monkeypatch.setattr(bench, "profile_entry", lambda v: None)
    assert bench.compute_roofline("f32_refine", 1, 1.0, 2000.0, 152) is None


def test_adi_flop_count_is_gated_on_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "adi.cu"
    src.write_text("adi v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"adi": {"fp64_ops_per_cell": 80.0, "fp64_flops_per_cell": 123.0,
                                                           "source_sha": bench.source_sha(str(src))}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SRC", {"adi": "adi.cu"})
    assert bench.adi_fp64_counts() == (80.0, 123.0)
    src.write_text("adi v2\n")
    assert bench.adi_fp64_counts() is None


def test_traffic_table_is_gated_on_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.source_sha(str(src))
    (prof / "traffic.json").write_text(json.dumps({"f64": {"dram_bytes_per_row": 60.0, "source_sha": sha,
                                                           "warp_inst_per_row": 2.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SRC", {"f64": "k.cu"})
    assert bench.traffic_per_row("f64") == 60.0
    assert bench.profile_entry("f64")["warp_inst_per_row"] == 2.0
    src.write_text("kernel v2\n")  # the kernel changed after the counters were taken
    assert bench.traffic_per_row("f64") is None
    assert bench.profile_entry("f64") is None

