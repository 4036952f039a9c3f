"""GPU parity of every entry point against the FP64 oracle, through the C ABI.

Sizes span several tiles with ragged tails; edge cases cover d = 1, k = 1,
k > n, unaligned d (scalar paths), planted ties, empty clusters, weights,
degenerate seeding and invalid labels.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import (COST_REL_F32, CENTROID_REL, assert_labels_match, centroid_err)

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ A1 / A0
@pytest.mark.parametrize("n,d", [(1, 1), (1037, 64), (999, 37), (300, 1030)])
def test_row_norms(gb, orc, n, d):
    X, _ = synth.gaussian_mixture(n, d, 5, seed=n + d)
    xn = H(gb.kmeans_row_norms(T(X)))
    ref = orc.row_norms(X)
    np.testing.assert_allclose(xn, ref, rtol=(d / 32 + 8) * 2.0 ** -24 * 2)


@pytest.mark.parametrize("n,d", [(513, 64), (77, 1030), (5, 3)])
@pytest.mark.parametrize("residuals", [False, True])
def test_quantize_bf16_bitexact(gb, orc, n, d, residuals):
    X, _ = synth.gaussian_mixture(n, d, 4, seed=7)
    X[0, 0] = 0.0
    Xq, _ = gb.kmeans_quantize(T(X), "bf16", residuals=residuals)
    got = H(Xq.view(torch.int16)).view(np.uint16)
    assert np.array_equal(got, orc.quant_bf16(X))


@pytest.mark.parametrize("n,d", [(513, 64), (77, 1030), (300, 37), (5, 3)])
def test_quantize_bf16_residuals_bound(gb, orc, n, d):
    """The rows' rounding residuals ||x - bf16(x)|| are upper bounds, above the exact value by no
    more than the FP32 summation margin the kernel adds, sqrt(1 + (d + 4) 2^-23) (1 + 2.4e-7)."""
    X, _ = synth.gaussian_mixture(n, d, 4, seed=8)
    X[1] = 0.0
    _, r = gb.kmeans_quantize(T(X), "bf16")
    xq = orc.bf16_to_f32(orc.quant_bf16(X)).astype(np.float64)
    exact = np.sqrt(((X.astype(np.float64) - xq) ** 2).sum(axis=1))
    got = H(r).astype(np.float64)
    assert np.all(got >= exact)
    margin = np.sqrt(1 + (d + 4) * 2.0 ** -23) * (1 + 2.4e-7) * (1 + 1e-6)
    assert np.all(got <= exact * margin + 1e-30)
    assert got[1] == 0.0


# one read of a block in a mapped host block (or on the device): the copy, norms, BF16 copy and
# residuals equal those of the separate kernels bitwise, and the oracle's
@pytest.mark.parametrize("n,d,offset", [(1037, 1024, 0), (999, 37, 0), (300, 1000, 0), (257, 64, 1),
                                        (1, 1, 0)])
def test_ingest_from_host_block(gb, orc, n, d, offset):
    X, _ = synth.gaussian_mixture(n, d, 5, seed=n + d)
    X[0, 0] = 0.0
    blk = gb.HostBlock((n * d + offset,))
    src = blk.tensor[offset:offset + n * d].view(n, d)   # offset 1: a source that is not 16-byte aligned
    src.copy_(torch.from_numpy(X))
    Xd, xn, Xq, r = gb.kmeans_ingest(src, device=DEV)
    gb.gbkm_sync()
    assert np.array_equal(H(Xd), X)
    assert np.array_equal(H(xn), H(gb.kmeans_row_norms(Xd)))
    Xq2, r2 = gb.kmeans_quantize(Xd, "bf16")
    assert np.array_equal(H(Xq.view(torch.int16)), H(Xq2.view(torch.int16)))
    assert np.array_equal(H(r), H(r2))
    assert np.array_equal(H(Xq.view(torch.int16)).view(np.uint16), orc.quant_bf16(X))
    np.testing.assert_allclose(H(xn), orc.row_norms(X), rtol=(d / 32 + 8) * 2.0 ** -24 * 2)
    del src
    blk.close()


def test_ingest_from_device_without_copy(gb, orc):
    X, _ = synth.gaussian_mixture(2000, 256, 5, seed=4)
    Xg = T(X)
    none, xn, Xq, r = gb.kmeans_ingest(Xg, copy=False)
    gb.gbkm_sync()
    assert none is None
    assert np.array_equal(H(xn), H(gb.kmeans_row_norms(Xg)))
    Xq2, r2 = gb.kmeans_quantize(Xg, "bf16")
    assert np.array_equal(H(Xq.view(torch.int16)), H(Xq2.view(torch.int16))) and np.array_equal(H(r), H(r2))


def test_ingest_rejects_other_host_memory(gb):
    """Pageable memory, page-locked memory the library did not hand out, and a range that runs past
    the end of a host block are refused before any launch."""
    n, d = 64, 32
    plain = torch.zeros((n, d), dtype=torch.float32)
    pinned = torch.zeros((n, d), dtype=torch.float32).pin_memory()
    blk = gb.HostBlock((n, d))
    lib, ctx = gb.load(), gb.default_context(torch.device(DEV))
    ctx.bind_stream()
    xn = torch.empty(2 * n, dtype=torch.float32, device=DEV)
    for ptr, rows in ((plain.data_ptr(), n), (pinned.data_ptr(), n), (blk.tensor.data_ptr(), n + 1),
                      (blk.tensor.data_ptr() + 4 * d, n)):
        rc = lib.kmeans_ingest(ctx.handle, ptr, rows, d, None, gb._ptr(xn), None, None)
        assert rc == gb.GBKM_EINVAL
    assert lib.kmeans_ingest(ctx.handle, blk.tensor.data_ptr(), n, d, None, gb._ptr(xn), None, None) == 0
    gb.gbkm_sync()
    assert lib.gbkm_host_free(plain.data_ptr()) == gb.GBKM_EINVAL
    blk.close()


@pytest.mark.parametrize("n,d", [(300, 64), (40, 128), (33, 200), (7, 5)])
def test_quantize_fp8_bitexact(gb, orc, n, d):
    X, _ = synth.gaussian_mixture(n, d, 4, seed=8)
    X[1] *= 1e-3
    X[2, :] = 0.0
    Xq, s = gb.kmeans_quantize(T(X), "fp8")
    q_ref, s_ref = orc.quant_e4m3(X, 128)
    assert np.array_equal(H(s), s_ref)
    assert np.array_equal(H(Xq), q_ref)


# ------------------------------------------------------------------ A4 + A5
ASSIGN_CASES = [
    (1037, 64, 10),     # several row tiles + tail, one N chunk
    (2500, 96, 130),    # three N chunks with a tail
    (999, 37, 17),      # unaligned d: scalar loads
    (50, 8, 200),       # k > n
    (300, 1, 3),        # d = 1
    (257, 33, 1),       # k = 1
]


@pytest.mark.parametrize("n,d,k", ASSIGN_CASES)
def test_assign_f32_simt(gb, orc, n, d, k):
    X, _ = synth.gaussian_mixture(n, d, max(2, k // 2), seed=n * 7 + k)
    C = synth.gaussian_mixture(k, d, max(2, k // 2), seed=n * 7 + k)[0] if k > 1 else X[:1].copy()
    Xg, Cg = T(X), T(C)
    min_d2 = torch.empty(n, dtype=torch.float32, device=DEV)
    nre = torch.zeros(1, dtype=torch.int64, device=DEV)
    lab = gb.kmeans_assign(Xg, Cg, engine="simt", min_d2=min_d2, n_rechecked=nre)
    gb.gbkm_sync()
    ref_lab, d1, d2, _ = assert_labels_match(orc, X, C.astype(np.float64), H(lab))
    md = H(min_d2)
    xn = orc.row_norms(X)
    scale = xn + (C.astype(np.float64) ** 2).sum(1).max()
    assert np.all(np.abs(md - d1) <= 1e-4 * scale + 1e-6)


def test_assign_planted_ties_resolved_exactly(gb, orc):
    """Points exactly midway between two centers, and duplicated centers: the exact rule picks
    the lowest index, and the recheck must reproduce it."""
    rng = np.random.default_rng(5)
    d, k = 48, 12
    C = rng.integers(-8, 8, size=(k, d)).astype(np.float32) * 2.0
    C[7] = C[3]                                     # duplicate center
    mids = []
    for a, b in [(0, 1), (2, 5), (4, 9), (6, 11)]:
        mids.append(0.5 * (C[a] + C[b]))            # exactly representable midpoints
    X = np.concatenate([np.stack(mids), C[3:4] + 0.25,
                        rng.normal(size=(400, d)).astype(np.float32) * 6]).astype(np.float32)
    nre = torch.zeros(1, dtype=torch.int64, device=DEV)
    lab = H(gb.kmeans_assign(T(X), T(C), engine="simt", n_rechecked=nre))
    ref, d1, d2 = orc.assign(X, C.astype(np.float64))
    assert np.array_equal(lab[:5], ref[:5])
    assert lab[4] == 3                               # duplicate: lower index
    assert int(H(nre)[0]) >= 5
    assert_labels_match(orc, X, C.astype(np.float64), lab)


def test_assign_recheck_off_still_valid(gb, orc):
    X, _ = synth.gaussian_mixture(2000, 64, 8, seed=3)
    C = X[:20].copy()
    lab = H(gb.kmeans_assign(T(X), T(C), engine="simt", recheck=False))
    ref, d1, d2 = orc.assign(X, C.astype(np.float64))
    gap = orc.near_tie_gap(X, d1, d2)
    assert np.all((lab == ref) | (gap < 1e-2))


# ------------------------------------------------------------------ A6 + A7
# k up to 2,048 takes the shared-memory label tables and the one-launch offsets; k above, the
# device-wide scan; d = 1,024 / 1,100 take 16 row loads in flight per thread, d = 64 / 1,030 eight
@pytest.mark.parametrize("n,d,k,weighted", [(3000, 64, 10, False), (2049, 37, 25, True),
                                            (600, 1030, 7, False), (5, 3, 9, True),
                                            (1500, 1100, 5, True), (900, 4, 3, False),
                                            (6000, 16, 2048, False), (7000, 24, 2049, True),
                                            (30000, 16, 3000, False), (2000, 1024, 40, False)])
def test_update_matches_oracle(gb, orc, n, d, k, weighted):
    X, z = synth.gaussian_mixture(n, d, k, seed=n + k)
    lab = (z % max(1, k - 2)).astype(np.int32)       # leaves empty clusters when k > 2
    C_old = synth.gaussian_mixture(k, d, k, seed=1 + n)[0]
    w = synth.integer_weights(n, seed=n) if weighted else None
    out = gb.kmeans_update(T(X), T(lab), T(C_old), w=T(w) if weighted else None)
    gb.gbkm_sync()
    ref = orc.update(X, lab, C_old.astype(np.float64), w=w)
    assert np.array_equal(H(out["counts"]), ref["N"])
    assert int(H(out["n_empty"])[0]) == ref["n_empty"]
    assert centroid_err(H(out["C_new"]), ref["C_new"], X, lab) <= CENTROID_REL
    empty = ref["N"] == 0
    assert np.array_equal(H(out["C_new"])[empty], C_old[empty])
    co, cn = float(H(out["cost_old"])[0]), float(H(out["cost_new"])[0])
    assert co == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
    assert cn == pytest.approx(ref["cost_new"], rel=COST_REL_F32)


@pytest.mark.parametrize("n,d,k,share", [(60_000, 96, 20, 0.85), (200_000, 33, 3, 0.999),
                                           (9_000, 1000, 4000, 0.6)])
def test_update_skewed_clusters(gb, orc, n, d, k, share):
    """One cluster holds most rows (its chunk sums span many 32-item runs of the fold), the rest are
    spread over the other clusters with some empty: counts, centroids and costs match the oracle."""
    rng = np.random.default_rng(n + k)
    X, _ = synth.gaussian_mixture(n, d, 5, seed=k)
    lab = rng.integers(0, max(1, k // 2), size=n).astype(np.int32)   # clusters >= k/2 stay empty
    big = rng.random(n) < share
    lab[big] = k // 3
    C_old = synth.gaussian_mixture(k, d, 3, seed=n)[0]
    out = gb.kmeans_update(T(X), T(lab), T(C_old))
    gb.gbkm_sync()
    ref = orc.update(X, lab, C_old.astype(np.float64))
    assert np.array_equal(H(out["counts"]), ref["N"])
    assert int(H(out["n_empty"])[0]) == ref["n_empty"]
    assert centroid_err(H(out["C_new"]), ref["C_new"], X, lab) <= CENTROID_REL
    empty = ref["N"] == 0
    assert np.array_equal(H(out["C_new"])[empty], C_old[empty])
    assert float(H(out["cost_old"])[0]) == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
    assert float(H(out["cost_new"])[0]) == pytest.approx(ref["cost_new"], rel=COST_REL_F32)


@pytest.mark.parametrize("k", [30, 3000])
def test_update_is_bit_reproducible(gb, k):
    X, z = synth.gaussian_mixture(20000, 128, k, seed=2)
    Xg, lg = T(X), T(z.astype(np.int32))
    C0 = T(np.zeros((k, 128), np.float32))
    a = gb.kmeans_update(Xg, lg, C0)
    A = (H(a["C_new"]).copy(), H(a["cost_new"]).copy())
    b = gb.kmeans_update(Xg, lg, C0)
    assert np.array_equal(A[0], H(b["C_new"])) and np.array_equal(A[1], H(b["cost_new"]))


def test_update_rejects_bad_labels(gb):
    X = T(np.ones((100, 4), np.float32))
    lab = torch.zeros(100, dtype=torch.int32, device=DEV)
    lab[17] = 5
    gb.kmeans_update(X, lab, T(np.zeros((3, 4), np.float32)))
    with pytest.raises(gb.GbkmError) as e:
        gb.gbkm_sync()
    assert e.value.code == gb.GBKM_EINVAL


@pytest.mark.parametrize("weighted", [False, True])
def test_cost_matches_oracle(gb, orc, weighted):
    X, _ = synth.gaussian_mixture(4099, 50, 9, seed=11)
    C = synth.gaussian_mixture(9, 50, 9, seed=12)[0]
    w = synth.integer_weights(4099, seed=4) if weighted else None
    cost = float(H(gb.kmeans_cost(T(X), T(C), w=T(w) if weighted else None))[0])
    assert cost == pytest.approx(orc.cost(X, C.astype(np.float64), w=w), rel=COST_REL_F32)


# ------------------------------------------------------------------ A3
@pytest.mark.parametrize("n,d,k,weighted", [(5000, 64, 10, False), (3001, 37, 20, True),
                                            (2048, 256, 33, False), (1, 4, 1, False)])
def test_seed_pp_matches_oracle(gb, orc, n, d, k, weighted):
    X, _ = synth.gaussian_mixture(n, d, max(1, k), seed=n + d)
    u = synth.seed_uniforms(k, seed=n)
    w = synth.integer_weights(n, seed=d) if weighted else None
    idx, C = gb.kmeans_seed_pp(T(X), k, T(u), w=T(w) if weighted else None)
    gb.gbkm_sync()
    ref_idx, ref_C, _, rc = orc.seed_pp(X, k, u, w=w)
    assert rc == 0
    assert np.array_equal(H(idx), ref_idx)
    assert np.array_equal(H(C), X[ref_idx])


@pytest.mark.parametrize("n,d,k,weighted", [(5000, 64, 10, False), (3000, 40, 20, True), (2048, 256, 33, False),
                                            (20000, 1024, 40, False)])
def test_seed_pp_with_bf16_copy_matches_oracle(gb, orc, n, d, k, weighted):
    """The variant that filters rows through the BF16 copy (kmeans_seed_pp_q) picks the same rows: the
    copy's lower bound only decides which rows need their FP32 distance."""
    X, _ = synth.gaussian_mixture(n, d, max(1, k), seed=n + d + 1)
    u = synth.seed_uniforms(k, seed=n + 1)
    w = synth.integer_weights(n, seed=d) if weighted else None
    Xg = T(X)
    Xq, xr = gb.kmeans_quantize(Xg, "bf16")
    idx, C = gb.kmeans_seed_pp(Xg, k, T(u), w=T(w) if weighted else None, Xq=Xq, xresid=xr)
    plain, _ = gb.kmeans_seed_pp(Xg, k, T(u), w=T(w) if weighted else None)
    gb.gbkm_sync()
    ref_idx, _, _, rc = orc.seed_pp(X, k, u, w=w)
    assert rc == 0
    assert np.array_equal(H(idx), ref_idx)
    assert torch.equal(idx, plain)
    assert np.array_equal(H(C), X[ref_idx])


def test_seed_pp_degenerate_reports(gb):
    X = np.repeat(np.array([[0.0, 0.0], [3.0, 4.0]], np.float32), 50, axis=0)
    idx, C = gb.kmeans_seed_pp(T(X), 3, T(np.array([0.1, 0.5, 0.5])))
    with pytest.raises(gb.GbkmError) as e:
        gb.gbkm_sync()
    assert e.value.code == gb.GBKM_EDEGENERATE
    got = H(idx)
    assert got[2] == -1 and got[0] >= 0 and got[1] >= 0


# ------------------------------------------------------------------ A2 (SIMT fallback shapes)
@pytest.mark.parametrize("n,d,r", [(700, 48, 6), (130, 100, 10)])
def test_project_simt_matches_oracle(gb, orc, n, d, r):
    X, _ = synth.gaussian_mixture(n, d, 5, seed=r)
    V = synth.orthonormal_basis(d, r, seed=r)
    Y, L = gb.kmeans_project_block(T(X), T(V.astype(np.float32)), lift=True)
    Yr, Lr = orc.project(X, V.astype(np.float32).astype(np.float64), lift=True)
    xn = np.sqrt(orc.row_norms(X))[:, None]
    assert np.all(np.abs(H(Y) - Yr) <= 1e-5 * xn + 1e-6)
    assert np.all(np.abs(H(L) - Lr) <= 1e-5 * xn + 1e-6)


# ------------------------------------------------------------------ Lloyd, stepwise parity
def test_lloyd_stepwise_parity_small_workload(gb, orc):
    """10,000 x 64, k = 10 (the small plain workload): seeding, then each Lloyd step checked
    against the oracle consuming the GPU's centers; cost non-increasing."""
    X, _ = synth.gaussian_mixture(10_000, 64, 10, seed=0)
    u = synth.seed_uniforms(10, seed=0)
    Xg = T(X)
    idx, C = gb.kmeans_seed_pp(Xg, 10, T(u))
    ref_idx, _, _, _ = orc.seed_pp(X, 10, u)
    assert np.array_equal(H(idx), ref_idx)
    prev = np.inf
    lab = torch.empty(10_000, dtype=torch.int32, device=DEV)
    for t in range(20):
        Ch = H(C).astype(np.float64)
        gb.kmeans_assign(Xg, C, engine="simt", labels=lab)
        L = H(lab)
        assert_labels_match(orc, X, Ch, L)
        out = gb.kmeans_update(Xg, lab, C)
        ref = orc.update(X, L, Ch)
        assert centroid_err(H(out["C_new"]), ref["C_new"], X, L) <= CENTROID_REL
        co, cn = float(H(out["cost_old"])[0]), float(H(out["cost_new"])[0])
        assert co == pytest.approx(ref["cost_old"], rel=COST_REL_F32)
        assert cn == pytest.approx(ref["cost_new"], rel=COST_REL_F32)
        assert co <= prev * (1 + 1e-12) and cn <= co * (1 + 1e-12)
        prev = cn
        C = out["C_new"]
