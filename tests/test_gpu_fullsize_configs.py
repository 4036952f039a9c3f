"""Parity at the full sizes of the streamed, batched and learned workloads, in the launch
configuration bench.py times.

Streamed block projection + assignment: 2,000,000 points in d = 2,048 (500-component mixture in a
random rank-64 subspace plus N(0, 0.1^2) noise), 31 chunks of 65,536 rows (the last 33,920),
projected to r = 64 by the BF16 projection with V = Q; every chunk's first 4,096 rows and the whole
tail chunk are checked against the FP64 projection.  Then k = 1,000 on all 2,000,000 coordinates:
k-means++ indices bit-identical to the oracle's, and one Lloyd step in BF16, FP8 and 3xTF32 with
every label checked against the FP64 full scan and the update against the FP64 CF sums.
Batched: a deterministic subset of the 512-problem list (every eighth problem, all three d values),
4 k-means++ seeds each, one iteration checked stepwise per (problem, seed).
Learned: k = 16,384 centers in d = 256, the learned assignment of a 65,536-row slice against the
FP64 full scan over all k.
The generators run in spawned processes (never forked after CUDA is up).
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import (CENTROID_REL, COST_REL_F32, TIE_REL, assert_labels_match, centroid_err)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

STREAM_N, STREAM_D, STREAM_R, STREAM_CHUNK, STREAM_K = 2_000_000, 2048, 64, 65536, 1000


def _stream_chunk(job):
    row0, rows = job
    Q = synth.orthonormal_basis(STREAM_D, STREAM_R, 0)
    X, _ = synth.subspace_mixture_chunk(Q, row0, rows, 500, 0)
    return row0, X


def _pool():
    return cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn"))


def test_stream_config_full_size(gb, orc):
    Q = synth.orthonormal_basis(STREAM_D, STREAM_R, 0)
    Vg = torch.from_numpy(Q.astype(np.float32)).to(DEV)
    Y = torch.empty((STREAM_N, STREAM_R), dtype=torch.float32, device=DEV)
    jobs = [(r0, min(STREAM_N, r0 + STREAM_CHUNK) - r0) for r0 in range(0, STREAM_N, STREAM_CHUNK)]
    assert len(jobs) == 31 and jobs[-1][1] == 33_920
    u8, d = 2.0 ** -8, STREAM_D
    with _pool() as ex:
        for row0, X in ex.map(_stream_chunk, jobs):
            rows = X.shape[0]
            Xg = torch.from_numpy(X).to(DEV)
            Xb, _ = gb.kmeans_quantize(Xg, "bf16", residuals=False)
            gb.kmeans_project_block(Xb, Vg, Y=Y[row0:row0 + rows])
            chk = rows if rows < STREAM_CHUNK else 4096
            Yc = Y[row0:row0 + chk].cpu().numpy()
            Yr = orc.project(X[:chk], Q.astype(np.float32).astype(np.float64))
            xn = np.sqrt(orc.row_norms(X[:chk]))[:, None]
            assert np.all(np.abs(Yc - Yr) <= (2 * u8 + d * 2.0 ** -22) * xn + 1e-5), row0
    gb.gbkm_sync()
    Yh = Y.cpu().numpy()
    u = synth.seed_uniforms(STREAM_K, seed=0)
    idx, C = gb.kmeans_seed_pp(Y, STREAM_K, torch.from_numpy(u).to(DEV))
    gb.gbkm_sync()
    ref_idx, _, _, rc = orc.seed_pp(Yh, STREAM_K, u)
    assert rc == 0 and np.array_equal(idx.cpu().numpy(), ref_idx)
    Ch = C.cpu().numpy().astype(np.float64)
    lab_or, d1, d2 = orc.assign(Yh, Ch)
    gap = orc.near_tie_gap(Yh, d1, d2)
    xn = gb.kmeans_row_norms(Y)
    Yb, Yr_ = gb.kmeans_quantize(Y, "bf16")
    Y8, s8 = gb.kmeans_quantize(Y, "fp8")
    for form, Xop, sc in (("bf16", Yb, Yr_), ("fp8", Y8, s8), ("f32", None, None)):
        lab = gb.kmeans_assign(Y, C, Xop=Xop, Xop_scales=sc, xnorm=xn, compute=form, engine="tcgen05")
        out = gb.kmeans_update(Y, lab, C)
        gb.gbkm_sync()
        L = lab.cpu().numpy()
        diff = L != lab_or
        assert not (diff & (gap >= TIE_REL)).any(), (form, int((diff & (gap >= TIE_REL)).sum()))
        if diff.any():
            rows = np.nonzero(diff)[0]
            dg = ((Yh[rows].astype(np.float64) - Ch[L[rows]]) ** 2).sum(1)
            assert np.all(dg <= d1[rows] * (1 + 2 * TIE_REL) + 1e-30), form
        ref = orc.update(Yh, L, Ch)
        assert np.array_equal(out["counts"].cpu().numpy(), ref["N"]), form
        assert centroid_err(out["C_new"].cpu().numpy(), ref["C_new"], Yh, L) <= CENTROID_REL, form
        assert float(out["cost_old"].item()) == pytest.approx(ref["cost_old"], rel=COST_REL_F32), form
        assert float(out["cost_new"].item()) == pytest.approx(ref["cost_new"], rel=COST_REL_F32), form


def _batch_problem(job):
    n, d, k, seed = job
    X, _ = synth.gaussian_mixture(n, d, k, seed=seed)
    return X


@pytest.mark.parametrize("compute", ["f32", "bf16"])
def test_batch_config_problem_list(gb, orc, compute):
    seeds = 4
    shapes = synth.batch_problem_list(512, seed=0)[::8]
    assert len(shapes) == 64 and {s["d"] for s in shapes} == {32, 128, 512}
    with _pool() as ex:
        Xs = list(ex.map(_batch_problem, [(s["n"], s["d"], s["k"], s["seed"]) for s in shapes]))
    probs, host = [], []
    for s, X in zip(shapes, Xs):
        U = np.stack([synth.seed_uniforms(s["k"], seed=s["seed"] * seeds + j) for j in range(seeds)])
        probs.append({"X": torch.from_numpy(X).to(DEV), "k": s["k"], "u": torch.from_numpy(U).to(DEV)})
        host.append((X, s["k"], U))
    gb.kmeans_batch_run(probs, seeds, 1, compute=compute, graph=True)
    gb.gbkm_sync()
    for pr, (X, k, U) in zip(probs, host):
        Cb, Lb, cb = pr["C_out"].cpu().numpy(), pr["labels_out"].cpu().numpy(), pr["cost_out"].cpu().numpy()
        for s in range(seeds):
            _, C0, _, rc = orc.seed_pp(X, k, U[s])
            assert rc == 0
            assert_labels_match(orc, X, C0, Lb[s])
            ref = orc.update(X, Lb[s], C0)
            assert centroid_err(Cb[s], ref["C_new"], X, Lb[s]) <= CENTROID_REL
            assert cb[s, 0] == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
            assert cb[s, 1] == pytest.approx(ref["cost_new"], rel=COST_REL_F32)


def test_learned_config_k16384_slice(gb, orc):
    from paper_1502_04265_gb300.learned import ProposalNet

    n, d, k, h, ntrain = 65_536, 256, 16_384, 256, 100_000
    Xall, _, prm = synth.gaussian_mixture(n + ntrain, d, k, seed=0, return_params=True)
    C = torch.from_numpy(np.ascontiguousarray(prm["mu"], np.float32)).to(DEV)
    Xg = torch.from_numpy(np.ascontiguousarray(Xall[:n])).to(DEV)
    Xtg = torch.from_numpy(np.ascontiguousarray(Xall[n:])).to(DEV)
    lt = gb.kmeans_assign(Xtg, C, compute="f32")
    net = ProposalNet(d, h, k, seed=0, device=DEV)
    Xtb, _ = gb.kmeans_quantize(Xtg, "bf16", residuals=False)
    net.train(Xtb, lt, epochs=3, batch=4096, lr=3e-3)
    s2 = gb.kmeans_center_separation(C)
    Xh, _ = gb.kmeans_quantize(Xg, "bf16", residuals=False)
    labels, nf = gb.kmeans_learned_assign(net, Xg, Xh, C, s2, topm=32)
    gb.gbkm_sync()
    assert_labels_match(orc, Xall[:n], prm["mu"].astype(np.float64), labels.cpu().numpy())
    assert 0 <= int(nf.item()) <= n
