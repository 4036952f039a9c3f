"""The replicated-run host logic of bench.py on two CPU ranks (gloo): the launcher's environment, the
barrier, the maximum of the step time over the ranks and the whole-job value; and the reference arm's
ranks other than 0, which exit without work or output."""
import json
import os
import socket
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch

    import bench

    r = bench.Ranks("gloo", torch.device("cpu"))
    # each rank's own step time; the line reports the slowest rank's
    ms = 10.0 + 5.0 * rank
    r.barrier()
    ms_max = r.max_over_ranks(ms)
    value = r.whole_job(1000.0, ms_max)
    r.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": r.world, "rank": r.rank, "ms_max": ms_max, "value": value}, f)
    r.close()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_work():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    with tempfile.TemporaryDirectory() as out:
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = [json.load(open(os.path.join(out, f"rank{r}.json"))) for r in range(world)]
    for r, e in enumerate(res):
        assert e["world"] == world and e["rank"] == r
        assert e["ms_max"] == 15.0                     # the slowest rank's time, on every rank
        assert e["value"] == pytest.approx(world * 1000.0 / 15e-3)  # all ranks' work in that time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import torch

    import bench

    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        r = bench.Ranks("gloo", torch.device("cpu"))
        assert (r.world, r.rank) == (1, 0)
        r.barrier()
        assert r.max_over_ranks(3.5) == 3.5
        assert r.whole_job(10.0, 2.0) == pytest.approx(5000.0)
    finally:
        os.environ.update(env)


def test_reference_arm_ranks_other_than_zero_exit_quietly():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "small", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
