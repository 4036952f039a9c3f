"""Parity at the full sizes of the workloads, in the configuration bench.py times.

High-dimensional workload: n = 200,000, d = 1,024, k = 100 (100-component mixture, seed 0).
The oracle checks seeding indices over the whole set, the labels of every row (an FP64 full scan,
OpenMP over the host cores) and the whole update step (FP64 CF sums over all rows).
Small workload: n = 10,000, d = 64, k = 10, 20 Lloyd iterations in every precision form.
StructuredWithNoise: 50 hidden sets x 5,000 points, d = 1,000, k = 50 (and an 8 x 500 instance).
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import COST_REL_F32, CENTROID_REL, assert_labels_match, centroid_err

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def highdim():
    X, _ = synth.gaussian_mixture(200_000, 1024, 100, seed=0)
    u = synth.seed_uniforms(100, seed=0)
    return X, u


def test_highdim_seeding_matches_oracle(gb, orc, highdim):
    """Both seeding calls (FP32 rows only, and with the BF16 copy as a filter) pick the oracle's rows."""
    X, u = highdim
    Xg = torch.from_numpy(X).to(DEV)
    ug = torch.from_numpy(u).to(DEV)
    idx, C = gb.kmeans_seed_pp(Xg, 100, ug)
    Xq, xr = gb.kmeans_quantize(Xg, "bf16")
    idx_q, _ = gb.kmeans_seed_pp(Xg, 100, ug, Xq=Xq, xresid=xr)
    gb.gbkm_sync()
    ref_idx, _, _, rc = orc.seed_pp(X, 100, u)
    assert rc == 0
    assert np.array_equal(idx.cpu().numpy(), ref_idx)
    assert np.array_equal(idx_q.cpu().numpy(), ref_idx)


@pytest.mark.parametrize("form", ["bf16", "f32"])
def test_highdim_lloyd_step_matches_oracle(gb, orc, highdim, form):
    X, u = highdim
    n, d, k = X.shape[0], X.shape[1], 100
    Xg = torch.from_numpy(X).to(DEV)
    _, C = gb.kmeans_seed_pp(Xg, k, torch.from_numpy(u).to(DEV))
    xn = gb.kmeans_row_norms(Xg)
    Xop = gb.kmeans_quantize(Xg, "bf16")[0] if form == "bf16" else None
    labels = torch.empty(n, dtype=torch.int32, device=DEV)
    for _ in range(3):  # a few iterations so that clusters are split and ties appear
        Ch = C.cpu().numpy().astype(np.float64)
        nre = torch.zeros(1, dtype=torch.int64, device=DEV)
        gb.kmeans_assign(Xg, C, Xop=Xop, xnorm=xn, compute=form, labels=labels, n_rechecked=nre)
        out = gb.kmeans_update(Xg, labels, C)
        gb.gbkm_sync()
        L = labels.cpu().numpy()
        assert_labels_match(orc, X, Ch, L)
        ref = orc.update(X, L, Ch)
        assert np.array_equal(out["counts"].cpu().numpy(), ref["N"])
        assert centroid_err(out["C_new"].cpu().numpy(), ref["C_new"], X, L) <= CENTROID_REL
        assert float(out["cost_old"].item()) == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
        assert float(out["cost_new"].item()) == pytest.approx(ref["cost_new"], rel=COST_REL_F32)
        C = out["C_new"]


@pytest.mark.parametrize("form,engine", [("f32", "simt"), ("f32", "tcgen05"), ("bf16", "auto"),
                                         ("fp8", "auto")])
def test_small_workload_full_run(gb, orc, form, engine):
    """10,000 x 64, k = 10: seeding + 20 iterations on the GPU in each precision form.  The seeding
    is bit-exact; the final state is checked stepwise (the oracle takes the GPU's centers); the
    independent oracle trajectory reaches the same cost up to near-tie drift."""
    from paper_1502_04265_gb300 import driver

    X, _ = synth.gaussian_mixture(10_000, 64, 10, seed=0)
    u = synth.seed_uniforms(10, seed=0)
    Xg = torch.from_numpy(X).to(DEV)
    out = driver.lloyd(Xg, 10, 20, torch.from_numpy(u).to(DEV), compute=form, engine=engine,
                       return_trace=True)
    gb.gbkm_sync()
    ref_idx, C0, _, _ = orc.seed_pp(X, 10, u)
    assert np.array_equal(out["seed_idx"].cpu().numpy(), ref_idx)
    C = out["C"].cpu().numpy().astype(np.float64)
    trace = out["trace"].cpu().numpy()
    assert np.all(np.diff(trace.reshape(-1)) <= 1e-9 * trace[0, 0])
    # stepwise parity at the final state: one more step from the GPU's centers on both sides
    Cg = out["C"]
    Xop, sc = gb.kmeans_quantize(Xg, form) if form in ("bf16", "fp8") else (None, None)
    lab = gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=sc, compute=form, engine=engine)
    step = gb.kmeans_update(Xg, lab, Cg)
    L = lab.cpu().numpy()
    assert_labels_match(orc, X, C, L)
    ref = orc.update(X, L, C)
    assert centroid_err(step["C_new"].cpu().numpy(), ref["C_new"], X, L) <= CENTROID_REL
    assert float(step["cost_old"].item()) == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
    assert float(step["cost_new"].item()) == pytest.approx(ref["cost_new"], rel=COST_REL_F32)
    # the independent oracle trajectory from the same seeds: the same local optimum up to the
    # drift a near-tie flip causes (trajectories are compared on cost only)
    ref_C, ref_L, ref_trace, _ = orc.lloyd(X, C0, 20)
    assert trace[-1, 1] == pytest.approx(ref_trace[-1], rel=1e-4)


@pytest.mark.parametrize("d", [64, 300, 320])
def test_auto_form_matches_f32(gb, d):
    """driver.lloyd(compute="auto") takes FP32 below 256 dimensions or where d % 8 != 0 (d = 300) and
    BF16 (certified recheck) otherwise (d = 320); both are exact, so the run matches the FP32 run
    from the same seeds."""
    from paper_1502_04265_gb300 import driver

    X, _ = synth.gaussian_mixture(20_000, d, 12, seed=d)
    u = torch.from_numpy(synth.seed_uniforms(12, seed=1)).to(DEV)
    Xg = torch.from_numpy(X).to(DEV)
    a = driver.lloyd(Xg, 12, 8, u, compute="auto", return_trace=True)
    b = driver.lloyd(Xg, 12, 8, u, compute="f32", return_trace=True)
    gb.gbkm_sync()
    assert torch.equal(a["seed_idx"], b["seed_idx"])
    same = float((a["labels"] == b["labels"]).float().mean().item())
    assert same >= 0.9999
    ta, tb = a["trace"].cpu().numpy(), b["trace"].cpu().numpy()
    assert abs(ta[-1, 1] - tb[-1, 1]) <= 1e-6 * tb[-1, 1]


@pytest.mark.parametrize("ell,y", [(8, 500), (50, 5000)])
@pytest.mark.parametrize("form", ["bf16", "f32"])
def test_structured_with_noise_matches_oracle(gb, orc, ell, y, form):
    """StructuredWithNoise (Section 3: ell hidden sets, 20 signal dimensions in [-10, 10], the rest in
    [-1/2, 1/2]), d = 1,000, k = ell: the seeding indices are exact, and three Lloyd steps from them
    (BF16 with the rows' residuals, as the bench runs it, or 3xTF32) give the oracle's labels on
    every row and its update."""
    d, k = 1000, ell
    X, _ = synth.structured_with_noise(ell, y, d, 20, seed=ell)
    n = X.shape[0]
    u = synth.seed_uniforms(k, seed=ell)
    Xg = torch.from_numpy(X).to(DEV)
    idx, C = gb.kmeans_seed_pp(Xg, k, torch.from_numpy(u).to(DEV))
    gb.gbkm_sync()
    ref_idx, _, _, rc = orc.seed_pp(X, k, u)
    assert rc == 0 and np.array_equal(idx.cpu().numpy(), ref_idx)
    xn = gb.kmeans_row_norms(Xg)
    Xop, Xr = gb.kmeans_quantize(Xg, "bf16") if form == "bf16" else (None, None)
    labels = torch.empty(n, dtype=torch.int32, device=DEV)
    for _ in range(3):
        Ch = C.cpu().numpy().astype(np.float64)
        gb.kmeans_assign(Xg, C, Xop=Xop, Xop_scales=Xr, xnorm=xn, compute=form, labels=labels)
        out = gb.kmeans_update(Xg, labels, C)
        gb.gbkm_sync()
        L = labels.cpu().numpy()
        assert_labels_match(orc, X, Ch, L)
        ref = orc.update(X, L, Ch)
        assert np.array_equal(out["counts"].cpu().numpy(), ref["N"])
        assert centroid_err(out["C_new"].cpu().numpy(), ref["C_new"], X, L) <= CENTROID_REL
        assert float(out["cost_old"].item()) == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
        assert float(out["cost_new"].item()) == pytest.approx(ref["cost_new"], rel=COST_REL_F32)
        C = out["C_new"]
