"""The compute-peak probes run on the GPU and give plausible figures (the roofline denominators
that the copy and cuBLAS measurements do not cover): positive, below twice the nominal dense
peaks of the part (BF16 2.25, TF32 1.1, FP8 4.5 PFLOP/s; FFMA 152 SMs x 128 lanes x 2 x 2.07 GHz),
and ordered as the units are (FP8 above BF16 above TF32; FP32 FMA above FP64 FMA)."""
import pytest

pytestmark = pytest.mark.gpu

NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp8": 4500.0, "ffma": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 152 * 64 * 2 * 2.07e9 / 1e12}


def test_probes_are_plausible(gb):
    ctx = gb.Context(0)
    got = {u: ctx.probe_peak(u) for u in NOMINAL}
    ctx.sync()
    for u, v in got.items():
        assert 0.0 < v < 2.0 * NOMINAL[u], (u, v)
    assert got["fp8"] > got["bf16"] > got["tf32"], got
    assert got["ffma"] > got["fp64"], got
    assert got["bf16"] > 0.3 * NOMINAL["bf16"], got
    ctx.close()
