"""The bench's reference arm (the FP64 oracle on the host cores) prints one JSON line with the
contract's keys, and the stored DRAM-traffic table it reports from is consistent; run on tiny
budgets, no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


@pytest.mark.parametrize("workload", ["small", "svd"])
def test_reference_arm_line(workload):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
           "--warmup", "3", "--cpu-seconds", "0.2"]
    if workload == "svd":
        cmd += ["--n", "2048", "--d", "256"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["higher_is_better"] is True and line["vs_baseline"] is None


def test_stored_traffic_entries_are_well_formed():
    """Every DRAM-traffic figure the bench may report names an ncu summary that exists under
    profiles/, kernel sources that exist, and a positive byte count; the lookup returns it only while
    those sources are unchanged (their hash is recomputed here, as the bench does)."""
    sys.path.insert(0, ROOT)
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(bench)
    finally:
        sys.argv = argv
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        table = json.load(f)
    assert table
    csrc = os.path.join(ROOT, "paper_1502_04265_gb300", "csrc")
    for key, e in table.items():
        assert e["dram_bytes_per_launch"] > 0, key
        assert os.path.exists(os.path.join(ROOT, e["capture"])), (key, e["capture"])
        assert all(os.path.exists(os.path.join(csrc, s)) for s in e["sources"]), key
        valid = e["source_hash"] == bench.source_hash(e["sources"])
        assert bench.stored_traffic(key) == (e["dram_bytes_per_launch"] if valid else None), key
