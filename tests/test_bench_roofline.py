"""The bench's roofline arithmetic: achieved = algorithmic bytes (or flops) per launch / average
launch time, frac = achieved / the measured peak of the bound unit, and each form's unit peak.
Host only, no GPU."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_roof", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "measured",
         "probed": {"tf32": 1200.0, "fp8": 3000.0, "ffma": 70.0, "fp64": 1.0}}


def test_hbm_bound_kernel(bench):
    r = bench.roofline(PEAKS, "segsum", 150e-6, 820e6, 0.0, 1000.0, 0.01, traffic=831e6)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6800.0
    assert r["achieved"] == pytest.approx(820e6 / 150e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["kernel_ms"] == pytest.approx(0.15) and r["traffic"] == 831e6
    assert r["peak_source"] == "measured (of measured)"


def test_bound_follows_the_larger_time(bench):
    # 1 MB against 10 TFLOP: the compute time dominates, so the kernel is judged against its unit
    r = bench.roofline(PEAKS, "gemm", 1e-2, 1e6, 10e12, 1000.0, 0.01)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == 1000.0
    assert r["achieved"] == pytest.approx(10e12 / 1e-2 / 1e12)
    alu = bench.roofline(PEAKS, "take", 1e-3, 1e9, 1e9, 1.0, 0.01, bound="alu")
    assert alu["bound"] == "alu" and alu["frac"] == pytest.approx(1e9 / 1e-3 / 1e12 / 1.0)


def test_unit_peaks_per_form(bench):
    short, long_ = 0.5, 5.0
    assert bench.unit_peak(PEAKS, "bf16", True, short) == 1900.0
    assert bench.unit_peak(PEAKS, "bf16", True, long_) == 1700.0          # sustained inside a long step
    assert bench.unit_peak(PEAKS, "fp8", True, short) == pytest.approx(max(1900.0 * 2.0, 3000.0))
    tf32 = max(1900.0 * 1.1 / 2.25, 1200.0)
    assert bench.unit_peak(PEAKS, "f32", True, short) == pytest.approx(tf32 / 3.0)  # three products
    assert bench.unit_peak(PEAKS, "f32", False, short) == pytest.approx(max(bench.FFMA_PEAK_TFLOPS, 70.0))
    assert bench.fp64_peak(PEAKS) == pytest.approx(max(bench.FP64_NOMINAL_TFLOPS, 1.0))


def test_fallback_peaks_are_labelled(bench):
    peaks = dict(PEAKS, source="fallback", probed=None)
    r = bench.roofline(peaks, "segsum", 1e-4, 1e8, 0.0, 1.0, 0.01)
    assert r["peak_source"] == "fallback (of fallback)"
    assert bench.unit_peak(peaks, "f32", True, 0.5) == pytest.approx(1900.0 * 1.1 / 2.25 / 3.0)
