"""The benchmark's roofline arithmetic (host logic, no GPU): each term's achieved rate is its
algorithmic work over the kernel time, its fraction that rate over the term's peak, its floor
the time the work would take at the peak; the binding term is the one with the largest floor;
the measured DRAM traffic is reported only for the kernel source it was measured on."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_binding_term_and_fractions():
    # 1e9 cells in 100 ms; 2e10 bytes at 1000 GB/s -> 20 ms floor; 100 FP32 inst per cell at
    # 10 T/s -> 10 ms; 10 SFU ops per cell at 0.25 T/s -> 40 ms: the SFU term binds
    counts = {"fp32_per_cell": 100.0, "sfu_per_cell": 10.0, "source": "test"}
    r = bench.roofline(100.0, 1e9, 2e10, counts, 10.0, 0.25, 1000.0, None, "k", 2000.0)
    t = r["terms"]
    assert t["hbm"]["achieved"] == pytest.approx(200.0) and t["hbm"]["frac"] == pytest.approx(0.2)
    assert t["alu"]["achieved"] == pytest.approx(1.0) and t["alu"]["frac"] == pytest.approx(0.1)
    assert t["sfu"]["achieved"] == pytest.approx(0.1) and t["sfu"]["frac"] == pytest.approx(0.4)
    assert t["hbm"]["floor_ms"] == pytest.approx(20.0)
    assert t["alu"]["floor_ms"] == pytest.approx(10.0)
    assert t["sfu"]["floor_ms"] == pytest.approx(40.0)
    assert r["binding_term"] == "sfu" and r["bound"] == "alu"        # SFU and FP32 are both ALU work
    assert r["frac"] == pytest.approx(0.4) and r["unit"] == "T SFU op/s"


def test_hbm_binds_without_op_counts():
    r = bench.roofline(50.0, 1e9, 1e11, None, 10.0, 1.0, 4000.0, 123, "k", 2000.0)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(1e11 / 0.05 / 1e9 / 4000.0, rel=1e-3)
    assert r["traffic"] == 123 and r["fp32_per_cell"] is None


def test_measured_traffic_only_for_its_kernel_source(monkeypatch):
    monkeypatch.setitem(bench.SWEEP_TRAFFIC, "kernels_sha256", bench.kernel_source_hash())
    monkeypatch.setitem(bench.SWEEP_TRAFFIC, "bytes_per_cell", {"single": 10.0})
    assert bench.measured_traffic("single", 1000) == 10000
    assert bench.measured_traffic("batched", 1000) is None
    monkeypatch.setitem(bench.SWEEP_TRAFFIC, "kernels_sha256", "0" * 16)
    assert bench.measured_traffic("single", 1000) is None
