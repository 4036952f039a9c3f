"""Pins of the weighted-insertion oracle (Section 2.1 clustering features, Section 2.3.1 weighted
BICO) against the direct definition of a feature's error and brute force over whole copies."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import bico as B


def _set(n, d, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, d)) * 3.0 + rng.normal(size=d), rng.integers(1, 6, size=n).astype(np.float64)


def test_cf_error_is_the_weighted_sum_of_squares():
    P, w = _set(40, 7, 1)
    N, S, Q = B.cf_of(P, w)
    mu = S / N
    direct = float((w * ((P - mu) ** 2).sum(axis=1)).sum())
    assert B.cf_error(N, S, Q) == pytest.approx(direct, rel=1e-12)
    assert B.cf_error(0.0, np.zeros(7), 0.0) == 0.0


@pytest.mark.parametrize("w", [1, 3, 17])
def test_error_increase_matches_adding_copies(w):
    """s w / (s + w) ||x - mu||^2 equals the error of the set with w copies of x added minus the
    error before (the derivation of Section 2.3.1), and never exceeds BICO's original estimate
    w ||x - mu||^2."""
    P, _ = _set(25, 5, 2)
    x = np.array([4.0, -1.0, 2.5, 0.5, 7.0])
    N, S, Q = B.cf_of(P)
    before = B.cf_error(N, S, Q)
    after = B.cf_error(*B.cf_of(np.vstack([P, np.repeat(x[None, :], w, axis=0)])))
    inc = B.error_increase(N, S / N, x, w)
    assert inc == pytest.approx(after - before, rel=1e-10)
    assert inc <= w * float(((x - S / N) ** 2).sum())


def _brute_insertable(s, c, T, d2, w):
    best = 0
    for k in range(int(w) + 1):
        if c + s * k / (s + k) * d2 <= T * (1 + 1e-12):
            best = k
    return best


@pytest.mark.parametrize("s,c,T,d2,w", [(10, 5.0, 20.0, 3.0, 50), (10, 5.0, 20.0, 1.0, 50), (3, 0.0, 9.0, 4.0, 7),
                                        (100, 99.0, 100.0, 0.5, 1000), (1, 0.0, 1.0, 100.0, 5), (8, 7.9, 8.0, 2.0, 3),
                                        (7, 32.0, 30.0, 120.0, 4)])
def test_insertable_is_the_largest_count_under_the_threshold(s, c, T, d2, w):
    got = B.insertable(s, c, T, d2, w)
    assert got == _brute_insertable(s, c, T, d2, w)
    if s * d2 - T + c <= 0:
        assert got == w


def test_nearest_reference_matches_cdist_with_lowest_index_ties():
    rng = np.random.default_rng(3)
    R = rng.integers(-3, 4, size=(12, 3)).astype(np.float64)
    R[5] = R[2]                      # duplicate reference: ties go to the lower index
    X = rng.integers(-3, 4, size=(200, 3)).astype(np.float64)
    j, d2 = B.nearest_reference(X, R)
    D = cdist(X, R, "sqeuclidean")
    assert np.array_equal(j, np.argmin(D, axis=1))
    assert np.allclose(d2, D.min(axis=1))
    assert not np.any(j == 5)


def test_batch_query_against_the_definitions():
    rng = np.random.default_rng(4)
    refs = rng.normal(size=(6, 4)) * 5
    feats = [cf_ for cf_ in (B.cf_of(refs[f] + rng.normal(size=(int(rng.integers(1, 9)), 4))) for f in range(6))]
    N = np.array([f[0] for f in feats]); S = np.array([f[1] for f in feats]); Q = np.array([f[2] for f in feats])
    X = rng.normal(size=(50, 4)) * 5
    w = rng.integers(1, 20, size=50).astype(np.float64)
    T = 30.0
    j, d2, take = B.batch_query(X, w, refs, N, S, Q, T)
    for i in range(50):
        f = int(np.argmin(((refs - X[i]) ** 2).sum(axis=1)))
        assert j[i] == f
        mu = S[f] / N[f]
        assert d2[i] == pytest.approx(float(((X[i] - mu) ** 2).sum()))
        c = B.cf_error(N[f], S[f], Q[f])
        assert take[i] == _brute_insertable(N[f], c, T, d2[i], w[i])
