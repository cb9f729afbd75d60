"""Host-side pieces of bench.py: the roofline object's arithmetic and the guard that
reports ncu DRAM traffic only for the sources and the workload it was captured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_captured_sources_and_workload(monkeypatch):
    terms = bench.NCU_TRAFFIC["terms"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, "digest", bench.kernel_source_digest())
    assert bench.ncu_traffic("tf32", "energy", terms) == bench.NCU_TRAFFIC[("tf32", "energy")]
    assert bench.ncu_traffic("tf32", "energy", 4 * terms) is None       # another workload
    assert bench.ncu_traffic("bf16x3", "energy", terms) is None          # not captured
    monkeypatch.setitem(bench.NCU_TRAFFIC, "digest", "0" * 16)           # sources changed since
    assert bench.ncu_traffic("tf32", "energy", terms) is None


def test_roofline_takes_the_slower_contraction_and_its_algorithmic_flops():
    peaks = {"bf16_tflops": 2000.0, "sm_max_mhz": 2070.0}
    terms = 1e10
    # energy: 4 flop per term over 0.05 ms; coefficients: 2 over 0.04 ms
    k = {"coeff": (2, 0.08), "energy": (2, 0.10), "prep": (2, 0.01), "finish": (2, 0.01)}
    r = bench.roofline("tf32", k, terms, peaks, "measured")
    assert r["kernel"] == "energy" and r["bound"] == "tensor"
    assert abs(r["achieved"] - 4 * terms / 0.05e-3 / 1e12) < 1e-6
    assert abs(r["peak"] - 1000.0) < 1e-9 and abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    r3 = bench.roofline("bf16x3", k, terms, peaks, "measured")
    assert abs(r3["peak"] - 2000.0 / 3) < 1e-9
    r32 = bench.roofline("fp32", k, terms, peaks, "measured")
    assert r32["bound"] == "alu" and abs(r32["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert bench.roofline("tf32", {"coeff": (0, 0.0), "energy": (0, 0.0)}, terms, peaks, "m") is None
