"""The bench's roofline arithmetic and its traffic lookup (CPU, no GPU)."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}


def test_tensor_class_takes_the_binding_view():
    # 2e12 FLOPs and 6e10 bytes in 100 ms: 20 TFLOP/s (1 % of 2000) and
    # 600 GB/s (10 % of 6000): bytes bind
    r = bench._roofline("k_linear_tc", 10, 100.0, 2e12, PEAKS, "test", 80.0, 1.0, nbytes=6e10)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(600.0)
    assert r["frac"] == pytest.approx(0.1)
    assert r["other_view"]["bound"] == "tensor"
    assert r["other_view"]["frac"] == pytest.approx(0.01)
    assert r["work_per_launch"] == pytest.approx(6e9)


def test_tensor_class_without_bytes_uses_the_tensor_peak():
    r = bench._roofline("k_linear_tc", 1, 10.0, 4e12, PEAKS, "test", 80.0, 1.0)
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(400.0)
    assert r["frac"] == pytest.approx(0.2)
    assert "other_view" not in r


def test_float64_and_memory_classes():
    r = bench._roofline("k_slater", 4, 1000.0, 5e11, PEAKS, "test", 80.0, 1.0)
    assert r["bound"] == "alu" and r["peak"] == 1.0
    assert r["frac"] == pytest.approx(0.5)
    m = bench._roofline("k_message", 4, 1.0, 3e9, PEAKS, "test", 80.0, 1.0)
    assert m["bound"] == "hbm" and m["achieved"] == pytest.approx(3000.0)


def test_class_without_work_has_no_roofline():
    r = bench._roofline("k_wgrad", 24, 16.0, 0.0, PEAKS, "test", 80.0, 1.0)
    assert r["bound"] is None and r["frac"] is None


def test_traffic_lookup_is_gated_on_the_source(tmp_path, monkeypatch):
    src = "paper_1909_08423_gb300/csrc/tc_gemm.cu"
    good = {"k_linear_tc": {"dram_bytes_per_work": 0.04, "source": src, "source_sha16": bench._sha16(
        os.path.join(ROOT, src)), "note": "capture"}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(good))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench._traffic_per_work("k_linear_tc") == (0.04, "capture")
    assert bench._traffic_per_work("k_filter")[0] is None
    good["k_linear_tc"]["source_sha16"] = "0" * 16
    f.write_text(json.dumps(good))
    v, why = bench._traffic_per_work("k_linear_tc")
    assert v is None and "changed" in why
