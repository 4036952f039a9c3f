"""Pins of the per-piece lift (Section 2.2 piecy, Section 2.3 on the growth of the intrinsic
dimension): rank per piece and overall, exactness on data inside each piece's subspace, and the
Eckart-Young error of each piece."""
import numpy as np
import pytest

from oracle import piecy as P
from oracle import rsvd as R
from paper_1502_04265_gb300 import synth


def _pieces(n_pieces, rows, d, r, seed):
    """Each piece drawn from its own rank-r subspace."""
    out = []
    for q in range(n_pieces):
        out.append(synth.planted_spectrum(rows, d, np.geomspace(30.0, 3.0, r), seed=seed + q))
    return np.vstack(out)


def test_each_piece_has_rank_l_and_the_total_grows_by_l_per_piece():
    d, ell, rows = 60, 5, 80
    X = _pieces(4, rows, d, 12, seed=1)
    Oms = [synth.gaussian_sketch(d, 16, seed=q).astype(np.float64) for q in range(4)]
    Y, bases = P.lift_pieces(X, rows, Oms, ell)
    for q in range(4):
        assert P.intrinsic_dimension(Y[q * rows:(q + 1) * rows]) == ell
        assert P.intrinsic_dimension(Y[:(q + 1) * rows]) == (q + 1) * ell   # random subspaces: no overlap
    assert Y.shape == X.shape


def test_lift_is_exact_inside_each_piece_subspace():
    """A piece of rank <= l is left unchanged by its projection."""
    d, ell, rows = 40, 6, 50
    X = _pieces(3, rows, d, 6, seed=5)
    Oms = [synth.gaussian_sketch(d, 16, seed=10 + q).astype(np.float64) for q in range(3)]
    Y, _ = P.lift_pieces(X, rows, Oms, ell)
    assert np.allclose(Y, X, atol=1e-9 * np.abs(X).max())


def test_each_piece_meets_eckart_young():
    d, ell, rows = 50, 4, 120
    rng = np.random.default_rng(7)
    X = _pieces(2, rows, d, 20, seed=9) + 0.01 * rng.standard_normal((2 * rows, d))
    Oms = [synth.gaussian_sketch(d, 20, seed=20 + q).astype(np.float64) for q in range(2)]
    Y, bases = P.lift_pieces(X, rows, Oms, ell)
    for q in range(2):
        Xq, Yq = X[q * rows:(q + 1) * rows], Y[q * rows:(q + 1) * rows]
        opt = float((np.linalg.svd(Xq, compute_uv=False)[ell:] ** 2).sum())
        err = float(((Xq - Yq) ** 2).sum())
        assert opt <= err <= 1.07 * opt
        assert err == pytest.approx(R.best_fit_error(Xq, bases[q]), rel=1e-10)


def test_ragged_last_piece():
    d, ell = 30, 3
    X = _pieces(2, 45, d, 8, seed=30)[:77]
    Oms = [synth.gaussian_sketch(d, 16, seed=40 + q).astype(np.float64) for q in range(2)]
    Y, bases = P.lift_pieces(X, 45, Oms, ell)
    assert len(bases) == 2 and P.intrinsic_dimension(Y[45:]) == ell
