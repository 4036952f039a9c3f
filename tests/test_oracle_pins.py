"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check uses something other than the oracle itself: hand-worked values
(tests/golden), textbook definitions evaluated with independent library
routines (scipy cdist, numpy bincount / matmul / SVD, torch dtype casts),
closed forms, invariants the paper states, and brute force on tiny inputs.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_1502_04265_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------- assign (Section 1)

def test_assign_hand_example(orc):
    g = _gold("lloyd_1d_hand.json")
    X = np.array(g["X"], np.float32)
    lab, d1, d2 = orc.assign(X, np.array(g["C0"]))
    assert lab.tolist() == g["labels"]
    assert d1.tolist() == g["d1"]
    assert d2.tolist() == g["d2"]


def test_assign_matches_cdist_full_scan(orc):
    X, _ = synth.gaussian_mixture(700, 37, 9, seed=3)
    C = synth.gaussian_mixture(13, 37, 4, seed=4)[0].astype(np.float64)
    lab, d1, d2 = orc.assign(X, C)
    D = cdist(X.astype(np.float64), C, "sqeuclidean")
    order = np.argsort(D, axis=1, kind="stable")
    assert np.array_equal(lab, order[:, 0])
    np.testing.assert_allclose(d1, D[np.arange(len(X)), order[:, 0]], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(d2, D[np.arange(len(X)), order[:, 1]], rtol=1e-12, atol=1e-9)


def test_assign_ties_lowest_index_and_k1(orc):
    X = np.array([[1.0, 2.0], [5.0, 5.0]], np.float32)
    C = np.array([[0.0, 0.0], [1.0, 2.0], [1.0, 2.0]])  # duplicated center
    lab, d1, d2 = orc.assign(X, C)
    assert lab[0] == 1 and d1[0] == 0.0 and d2[0] == 0.0
    lab, d1, d2 = orc.assign(X, C[:1])
    assert lab.tolist() == [0, 0] and np.all(np.isinf(d2))
    # equidistant point: tie broken to the lower index
    lab, _, _ = orc.assign(np.array([[0.0, 1.0]], np.float32), np.array([[0.0, 2.0], [0.0, 0.0]]))
    assert lab[0] == 0


# --------------------------------------------------------------------------- update (Sections 1, 2, 2.1)

def test_update_hand_example(orc):
    g = _gold("lloyd_1d_hand.json")
    X = np.array(g["X"], np.float32)
    u = orc.update(X, np.array(g["labels"], np.int32), np.array(g["C0"]))
    assert u["N"].tolist() == g["N"]
    assert u["S"].tolist() == g["S"]
    assert u["Q"].tolist() == g["Q"]
    assert u["C_new"].tolist() == g["C1"]
    assert u["cost_old"] == g["cost_old"] and u["cost_new"] == g["cost_new"]


def test_update_matches_bincount_means(orc):
    X, z = synth.gaussian_mixture(2000, 19, 7, seed=5)
    k = 9  # two clusters stay empty
    lab = (z % 7).astype(np.int32)
    C_old = np.arange(k * 19, dtype=np.float64).reshape(k, 19)
    u = orc.update(X, lab, C_old)
    Xd = X.astype(np.float64)
    cnt = np.bincount(lab, minlength=k).astype(np.float64)
    for t in range(19):
        s = np.bincount(lab, weights=Xd[:, t], minlength=k)
        np.testing.assert_allclose(u["S"][:, t], s, rtol=1e-13, atol=1e-10)
        nz = cnt > 0
        np.testing.assert_allclose(u["C_new"][nz, t], s[nz] / cnt[nz], rtol=1e-13)
    assert np.array_equal(u["N"], cnt)
    assert u["n_empty"] == 2
    np.testing.assert_array_equal(u["C_new"][7:], C_old[7:])  # empty -> previous center
    q = np.bincount(lab, weights=(Xd * Xd).sum(1), minlength=k)
    np.testing.assert_allclose(u["Q"], q, rtol=1e-13)


def test_centroid_is_optimal_center(orc):
    """Section 1: for each subset the centroid is the optimal center -> no perturbation lowers the cost."""
    X, z = synth.gaussian_mixture(300, 6, 4, seed=8)
    lab = z.astype(np.int32)
    C_old = np.zeros((4, 6))
    u = orc.update(X, lab, C_old)
    Xd = X.astype(np.float64)

    def cost_fixed_labels(C):
        return float(((Xd - C[lab]) ** 2).sum())

    base = cost_fixed_labels(u["C_new"])
    for j in range(4):
        for t in range(6):
            for h in (1e-3, -1e-3, 0.5, -0.5):
                C = u["C_new"].copy()
                C[j, t] += h
                # exact increase is N_j h^2 (Section 2.1 identity); must be positive
                assert cost_fixed_labels(C) > base
                assert abs(cost_fixed_labels(C) - base - u["N"][j] * h * h) <= 1e-7 * base


def test_cf_identity_matches_direct_cost(orc):
    """Section 2.1: sum ||x-c||^2 = |P| ||mu-c||^2 + sum ||x-mu||^2, evaluated from the CF sums."""
    X, z = synth.gaussian_mixture(1500, 33, 5, seed=9)
    w = synth.integer_weights(1500, seed=9)
    C_old = synth.gaussian_mixture(5, 33, 5, seed=10)[0].astype(np.float64)
    lab, _, _ = orc.assign(X, C_old)
    u = orc.update(X, lab, C_old, w=w)
    Xd = X.astype(np.float64)
    direct_old = float((w * ((Xd - C_old[lab]) ** 2).sum(1)).sum())
    direct_new = float((w * ((Xd - u["C_new"][lab]) ** 2).sum(1)).sum())
    assert u["cost_old"] == pytest.approx(direct_old, rel=1e-12)
    assert u["cost_new"] == pytest.approx(direct_new, rel=1e-12)
    assert orc.cost_cf(u["N"], u["S"], u["Q"], C_old) == pytest.approx(direct_old, rel=1e-10)
    assert orc.cost_cf(u["N"], u["S"], u["Q"], u["C_new"]) == pytest.approx(direct_new, rel=1e-10)
    # the new cost from the CFs alone: sum_j Q_j - ||S_j||^2 / N_j
    nz = u["N"] > 0
    alt = float((u["Q"][nz] - (u["S"][nz] ** 2).sum(1) / u["N"][nz]).sum())
    assert alt == pytest.approx(direct_new, rel=1e-10)


def test_integer_weights_equal_replicated_points(orc):
    """Section 2.3 / footnote on integral weights: weight w acts as w copies of the point."""
    X, _ = synth.gaussian_mixture(120, 5, 3, seed=11)
    w = synth.integer_weights(120, seed=11, max_w=4)
    C = synth.gaussian_mixture(3, 5, 3, seed=12)[0].astype(np.float64)
    Xr = np.repeat(X, w.astype(int), axis=0)
    lab, _, _ = orc.assign(X, C)
    labr, _, _ = orc.assign(Xr, C)
    assert np.array_equal(np.repeat(lab, w.astype(int)), labr)
    a = orc.update(X, lab, C, w=w)
    b = orc.update(Xr, labr, C)
    np.testing.assert_allclose(a["C_new"], b["C_new"], rtol=1e-12)
    np.testing.assert_allclose(a["N"], b["N"])
    assert a["cost_new"] == pytest.approx(b["cost_new"], rel=1e-12)
    assert orc.cost(X, C, w=w) == pytest.approx(orc.cost(Xr, C), rel=1e-12)


# --------------------------------------------------------------------------- cost (Section 1)

def test_cost_matches_cdist_min(orc):
    X, _ = synth.gaussian_mixture(500, 12, 6, seed=13)
    C = synth.gaussian_mixture(6, 12, 6, seed=14)[0].astype(np.float64)
    w = synth.integer_weights(500, seed=13)
    D = cdist(X.astype(np.float64), C, "sqeuclidean")
    assert orc.cost(X, C) == pytest.approx(D.min(1).sum(), rel=1e-12)
    assert orc.cost(X, C, w=w) == pytest.approx((w * D.min(1)).sum(), rel=1e-12)


# --------------------------------------------------------------------------- Lloyd (Section 1)

def test_lloyd_cost_monotone(orc):
    X, _ = synth.gaussian_mixture(3000, 16, 12, seed=15)
    u = synth.seed_uniforms(12, seed=15)
    idx, C0, _, rc = orc.seed_pp(X, 12, u)
    assert rc == 0
    C, lab, trace, conv = orc.lloyd(X, C0, 15)
    assert np.all(np.diff(trace) <= 1e-9 * trace[0])


def test_bruteforce_hand_optimum():
    from oracle import bruteforce

    X = np.array([[0.0], [1.0], [10.0], [11.0], [20.0], [21.0]])
    best, lab, cents = bruteforce.optimum(X, 3)
    assert best == pytest.approx(1.5)  # three pairs, each 2 * 0.5^2
    assert sorted(cents[:, 0].tolist()) == [0.5, 10.5, 20.5]


@pytest.mark.parametrize("seed", range(6))
def test_lloyd_against_bruteforce_optimum(orc, seed):
    from oracle import bruteforce

    rng = np.random.default_rng(seed)
    n, k = int(rng.integers(5, 11)), int(rng.integers(2, 4))
    X = rng.normal(size=(n, 2)).astype(np.float32) * 3
    best, lab, cents = bruteforce.optimum(X, k)
    # optimal centroids are a fixed point of Lloyd and reach the optimum
    C, lab2, trace, _ = orc.lloyd(X, cents, 3)
    np.testing.assert_allclose(C, cents, rtol=1e-12, atol=1e-12)
    assert orc.cost(X, C) == pytest.approx(best, rel=1e-12)
    # any k-means++ start ends no better than the optimum
    idx, C0, _, rc = orc.seed_pp(X, k, synth.seed_uniforms(k, seed))
    C, _, trace, _ = orc.lloyd(X, C0, 20)
    assert orc.cost(X, C) >= best * (1 - 1e-12)


# --------------------------------------------------------------------------- k-means++ (Section 1)

def test_pp_pick_hand_intervals(orc):
    g = _gold("pp_pick_hand.json")
    D2 = np.array(g["D2"])
    for c in g["cases"]:
        assert orc.pp_pick(D2, c["u"]) == c["idx"], c
    w = np.array(g["weighted"]["w"])
    for c in g["weighted"]["cases"]:
        assert orc.pp_pick(D2, c["u"], w=w) == c["idx"], c
    assert orc.pp_pick(np.zeros(4), 0.3) is None


def test_pp_pick_interval_law(orc):
    """P(i) = w_i D2_i / sum: the u-interval of index i has exactly that length."""
    rng = np.random.default_rng(21)
    D2 = rng.exponential(size=40)
    D2[rng.integers(0, 40, 6)] = 0.0
    w = rng.integers(1, 4, size=40).astype(np.float64)
    p = w * D2
    P = np.cumsum(p)
    T = P[-1]
    for i in np.nonzero(p > 0)[0]:
        lo = (P[i - 1] if i > 0 else 0.0) / T
        hi = P[i] / T
        assert orc.pp_pick(D2, 0.5 * (lo + hi), w=w) == i


def test_seed_pp_structure(orc):
    X, _ = synth.gaussian_mixture(800, 10, 8, seed=22)
    u = synth.seed_uniforms(8, seed=22)
    idx, C, D2, rc = orc.seed_pp(X, 8, u)
    assert rc == 0
    assert idx[0] == int(np.floor(u[0] * 800))
    assert len(set(idx.tolist())) == 8
    np.testing.assert_array_equal(C, X[idx].astype(np.float64))
    Dall = cdist(X.astype(np.float64), X[idx].astype(np.float64), "sqeuclidean").min(1)
    np.testing.assert_allclose(D2, Dall, rtol=1e-12, atol=1e-12)
    assert np.all(D2[idx] == 0)
    # every later pick is the pp_pick of the D2 before it (replay with numpy D2)
    D = cdist(X.astype(np.float64), X[idx[:1]].astype(np.float64), "sqeuclidean")[:, 0]
    for j in range(1, 8):
        assert orc.pp_pick(D, u[j]) == idx[j]
        D = np.minimum(D, cdist(X.astype(np.float64), X[idx[j]:idx[j] + 1].astype(np.float64),
                                "sqeuclidean")[:, 0])
        D[idx[j]] = 0.0


def test_seed_pp_second_center_law_chi2(orc):
    """Empirical law of the second center vs D2/sum D2 (chi-square, fixed first center)."""
    from scipy.stats import chisquare

    rng = np.random.default_rng(23)
    X = rng.normal(size=(12, 3)).astype(np.float32)
    draws = 6000
    U = rng.random((draws, 2))
    U[:, 0] = 0.0  # first center is row 0
    counts = np.zeros(12)
    for t in range(draws):
        idx, _, _, rc = orc.seed_pp(X, 2, U[t])
        counts[idx[1]] += 1
    D2 = ((X.astype(np.float64) - X[0].astype(np.float64)) ** 2).sum(1)
    expected = D2 / D2.sum() * draws
    m = expected > 0
    assert counts[~m].sum() == 0
    assert chisquare(counts[m], expected[m]).pvalue > 1e-3


def test_seed_pp_weighted_first_center_and_degenerate(orc):
    X = np.array([[0.0], [0.0], [5.0], [5.0]], np.float32)
    w = np.array([1.0, 1.0, 3.0, 1.0])
    # prefix of w: 1, 2, 5, 6; u0 = 0.3 -> t = 1.8 -> index 1; u0 = 0.4 -> t = 2.4 -> index 2
    idx, _, _, rc = orc.seed_pp(X, 2, np.array([0.3, 0.5]), w=w)
    assert idx[0] == 1 and idx[1] in (2, 3)
    idx, _, _, rc = orc.seed_pp(X, 2, np.array([0.4, 0.5]), w=w)
    assert idx[0] == 2 and idx[1] in (0, 1)
    # k larger than the number of distinct points -> degenerate status
    idx, _, _, rc = orc.seed_pp(X, 3, np.array([0.0, 0.5, 0.5]))
    assert rc == -6


# --------------------------------------------------------------------------- projection (Section 2.2)

def test_project_matches_matmul_and_lift(orc):
    X, _ = synth.gaussian_mixture(200, 48, 5, seed=30)
    V = synth.orthonormal_basis(48, 6, seed=30)
    Y, L = orc.project(X, V, lift=True)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(Y, Xd @ V, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(L, Xd @ V @ V.T, rtol=1e-10, atol=1e-9)
    assert np.linalg.norm(Y) <= np.linalg.norm(Xd) * (1 + 1e-12)


def test_project_eckart_young(orc):
    """Projection onto the top-r right singular vectors leaves residual sum_{i>r} sigma_i^2."""
    rng = np.random.default_rng(31)
    X = (rng.normal(size=(300, 40)) @ np.diag(np.linspace(5, 0.1, 40))).astype(np.float32)
    Xd = X.astype(np.float64)
    _, s, Vt = np.linalg.svd(Xd, full_matrices=False)
    r = 7
    Y, L = orc.project(X, Vt[:r].T, lift=True)
    resid = np.linalg.norm(Xd - L) ** 2
    assert resid == pytest.approx((s[r:] ** 2).sum(), rel=1e-9)


def test_project_in_span_preserves_distances(orc):
    Q = synth.orthonormal_basis(64, 8, seed=32)
    rng = np.random.default_rng(32)
    Z = rng.normal(size=(50, 8)) * 4
    X = (Z @ Q.T).astype(np.float32)
    Y, L = orc.project(X, Q, lift=True)
    np.testing.assert_allclose(L, X, atol=1e-5)
    Dx = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    Dy = cdist(Y, Y, "sqeuclidean")
    np.testing.assert_allclose(Dy, Dx, rtol=1e-5, atol=1e-4)


# --------------------------------------------------------------------------- precision forms (no paper counterpart)

def test_bf16_matches_torch_cast(orc):
    import torch

    rng = np.random.default_rng(40)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32) * 37,
                        np.array([0.0, -0.0, 1.0, 65504.0, 3.0e38, 1e-40], np.float32)])
    bits = orc.quant_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(bits, ref)


def test_e4m3_matches_torch_cast(orc):
    import torch

    rng = np.random.default_rng(41)
    X = (rng.normal(size=(17, 300)) * rng.uniform(0.01, 50, size=(17, 1))).astype(np.float32)
    X[3, :128] = 0.0
    q, s = orc.quant_e4m3(X, block=128)
    nb = s.shape[1]
    for i in range(X.shape[0]):
        for b in range(nb):
            blk = X[i, b * 128:(b + 1) * 128].astype(np.float64)
            amax = np.abs(blk).max()
            sc = float(s[i, b])
            assert sc == 2.0 ** np.round(np.log2(sc))
            if amax > 0:
                assert amax / sc <= 448.0 and amax / (sc / 2) > 448.0
            ref = torch.from_numpy((blk / sc).astype(np.float32)).to(torch.float8_e4m3fn)
            ref = ref.view(torch.uint8).numpy()
            assert np.array_equal(q[i, b * 128:(b + 1) * 128], ref)
    # decode: x ~ scale * value within half an E4M3 step (relative 2^-4)
    dec = orc.e4m3_decode(q) * np.repeat(s, 128, axis=1)[:, :300]
    big = np.abs(X) > np.repeat(s, 128, axis=1)[:, :300] * 2.0 ** -6
    assert np.all(np.abs(dec - X)[big] <= np.abs(X)[big] * 2.0 ** -4 + 1e-30)


# --------------------------------------------------------------------------- row norms (Section 2.1)

def test_row_norms_hand_example(orc):
    """Hand-worked ||x||^2, including 2^32 + 1, which an FP32 accumulator would round to 2^32."""
    g = _gold("row_norms_hand.json")
    assert orc.row_norms(np.array(g["X"], np.float32)).tolist() == g["norms"]


def test_row_norms_match_einsum(orc):
    X, _ = synth.gaussian_mixture(3000, 257, 6, seed=41)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(orc.row_norms(X), np.einsum("ij,ij->i", Xd, Xd), rtol=1e-13, atol=0)
    assert orc.row_norms(X[:0]).shape == (0,)


# --------------------------------------------------------------------------- near-tie gap (the certified-tie rule)

def _num(v):
    return float("inf") if v == "inf" else float(v)


def test_near_tie_gap_hand_cases(orc):
    g = _gold("near_tie_gap_hand.json")
    for c in g["cases"]:
        got = orc.near_tie_gap(np.array([c["x"]], np.float32), np.array([_num(c["d1"])]),
                               np.array([_num(c["d2"])]))[0]
        want = _num(c["gap"])
        if np.isinf(want):
            assert np.isinf(got) and got > 0, c
        else:
            assert got == pytest.approx(want, rel=1e-15, abs=0), c


def test_parity_checker_excuses_only_certified_ties(orc):
    """A GPU label that picks the second-nearest center is excused only when the oracle's relative
    top-2 gap is below 1e-5: planted points at gap 5e-6 pass, at 2e-5 (and exactly 1e-5) they fail."""
    from parity_util import TIE_REL, assert_labels_match

    C = np.array([[0.0, 0.0], [1000.0, 0.0]])

    def planted(gap):
        # x on the segment's perpendicular offset: d1 = a^2 + h^2, d2 = (1000 - a)^2 + h^2, with a set
        # so that (d2 - d1) / d1 = gap, computed in FP64 and checked against the oracle's own gap
        h = 300.0
        lo, hi = 0.0, 500.0
        for _ in range(200):
            a = 0.5 * (lo + hi)
            d1, d2 = a * a + h * h, (1000.0 - a) ** 2 + h * h
            if (d2 - d1) / d1 > gap:
                lo = a
            else:
                hi = a
        return np.array([[a, h]], np.float32)

    for gap, excused in [(5e-6, True), (2e-5, False), (4e-4, False)]:
        X = planted(gap)
        lab, d1, d2 = orc.assign(X, C)
        real = orc.near_tie_gap(X, d1, d2)[0]
        assert lab[0] == 0 and (real < TIE_REL) == excused, (gap, real)
        wrong = np.array([1], np.int32)    # the second-nearest center
        if excused:
            assert_labels_match(orc, X, C, wrong)
        else:
            with pytest.raises(AssertionError):
                assert_labels_match(orc, X, C, wrong)
