"""Pins of the randomised-SVD oracle (Section 2.2, Section 2.3.2, Section 3's error measure)
against facts it does not compute itself: exact recovery of a planted low-rank spectrum, the
Eckart-Young optimum of the full SVD, and the matrix of replicated rows."""
import numpy as np
import pytest

from oracle import rsvd as R
from paper_1502_04265_gb300 import synth


def test_exact_low_rank_recovery():
    """rank(A) = 12 <= s: range(A Omega) = range(A), so the scheme is exact: the planted singular
    values and right singular vectors come back."""
    sig = np.geomspace(50.0, 2.0, 12)
    A = synth.planted_spectrum(300, 90, sig, seed=1)
    W = synth.orthonormal_basis(90, 12, 4)           # the planted right singular vectors
    Om = synth.gaussian_sketch(90, 16, seed=2)
    V, s = R.rsvd(A, Om, 8)
    np.testing.assert_allclose(s, sig[:8], rtol=1e-10)
    assert R.projector_distance(V, W[:, :8]) < 1e-9
    assert np.allclose(V.T @ V, np.eye(8), atol=1e-12)


def test_eckart_young_near_optimal():
    """Decaying spectrum plus a noise floor: the error measure is never below the full SVD's
    optimum (Eckart-Young) and stays within the 7% the paper reports for its redSVD runs (1.3% here
    with 16 oversampling columns)."""
    rng = np.random.default_rng(5)
    sig = 30.0 * 0.85 ** np.arange(60)
    A = synth.planted_spectrum(800, 200, sig, seed=3) + 0.01 * rng.standard_normal((800, 200))
    Om = synth.gaussian_sketch(200, 36, seed=6)
    V, s = R.rsvd(A, Om, 20)
    Vx, sx = R.exact_top(A, 20)
    e, e_opt = R.best_fit_error(A, V), R.best_fit_error(A, Vx)
    assert e_opt == pytest.approx(float((np.linalg.svd(A, compute_uv=False)[20:] ** 2).sum()), rel=1e-10)
    assert e_opt <= e <= 1.07 * e_opt
    # singular values of Q^T A' never exceed those of A' (Q has orthonormal columns) and the
    # leading ones are captured to 1% (0.05% for the first: the slow 0.85 decay leaves the last
    # of the 20 at 19% below)
    assert np.all(s <= sx * (1 + 1e-12))
    np.testing.assert_allclose(s[:10], sx[:10], rtol=1e-2)
    assert s[0] == pytest.approx(sx[0], rel=1e-3)


def test_weighted_rows_equal_replicated_rows():
    """Section 2.3.2: rows scaled by sqrt(w_i) have the best-fit subspace and singular values of
    the matrix holding w_i copies of each row."""
    sig = np.geomspace(20.0, 1.0, 10)
    A = synth.planted_spectrum(150, 40, sig, seed=7)
    w = synth.integer_weights(150, seed=8, max_w=4).astype(np.float64)
    F = np.repeat(A, w.astype(np.int64), axis=0)
    Vf, sf = R.exact_top(F, 6)
    Om = synth.gaussian_sketch(40, 16, seed=9)
    V, s = R.rsvd(A, Om, 6, w=w)
    np.testing.assert_allclose(s, sf, rtol=1e-10)
    assert R.projector_distance(V, Vf) < 1e-9
    # without the weights the subspace is a different one
    V0, _ = R.rsvd(A, Om, 6)
    assert R.projector_distance(V0, Vf) > 1e-3


def test_sign_normalised_and_projector_distance():
    V = np.array([[0.6, -0.8], [-0.8, -0.6], [0.0, 0.0]])
    N = R.sign_normalised(V)
    assert np.array_equal(N[:, 0], [-0.6, 0.8, 0.0]) and np.array_equal(N[:, 1], [0.8, 0.6, 0.0])
    assert R.projector_distance(V, N) < 1e-15
    e = np.eye(3)
    assert R.projector_distance(e[:, :1], e[:, 1:2]) == pytest.approx(1.0)
