"""GPU parity of per-piece bases with the d-dimensional lift (Section 2.2, piecy; Section 2.3 on the
intrinsic dimension every piece adds) against oracle/piecy.py, through the C ABI.

Data: five pieces (the last one ragged), each a mixture inside its own random rank-ell subspace of
R^d plus N(0, 0.01^2) noise, so that the singular values of a piece drop by orders of magnitude
after ell: the best-fit subspace of every piece is well separated and the GPU's basis (FP32 sums,
FP64 factorisations) and the oracle's (FP64) span the same space to ~1e-6 (Davis-Kahan: the
perturbation over the gap).  The same random matrix per piece goes to both sides.
Checks: per piece the sine of the largest principal angle between the two bases; every lifted row
against the oracle's within that sine (plus 1e-5 for the FP32 products) times ||x||; the numerical
rank of the first q pieces' lifted rows is q * ell (each piece adds ell dimensions); and per piece
the error ||A_q - lift(A_q)||_F^2 sits at the full SVD's optimum (Eckart-Young), as the paper's
Section 3 measures it.
"""
import numpy as np
import pytest
import torch

from oracle import piecy as OP
from oracle import rsvd as OR
from paper_1502_04265_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _pieces(d, ell, piece_rows, n, seed):
    parts = []
    for q, r0 in enumerate(range(0, n, piece_rows)):
        rows = min(piece_rows, n - r0)
        Qb = synth.orthonormal_basis(d, ell, seed=seed * 100 + q)
        Xq, _ = synth.subspace_mixture_chunk(Qb, 0, rows, 6, seed=seed * 100 + q, noise=0.01)
        parts.append(Xq)
    return np.concatenate(parts).astype(np.float32)


@pytest.mark.parametrize("d,ell,s,piece_rows,n,weighted", [(256, 16, 32, 1000, 4600, False),
                                                           (512, 32, 48, 2048, 7000, True),
                                                           (200, 10, 16, 700, 2100, False)])
def test_piecy_lift_matches_oracle(gb, d, ell, s, piece_rows, n, weighted):
    X = _pieces(d, ell, piece_rows, n, seed=d)
    pieces = (n + piece_rows - 1) // piece_rows
    Om = np.stack([synth.gaussian_sketch(d, s, seed=1000 + q) for q in range(pieces)])
    w = synth.integer_weights(n, seed=d) if weighted else None
    L, V, sig, info = gb.kmeans_piecy_lift(T(X), piece_rows, T(Om), ell, w=None if w is None else T(w))
    gb.gbkm_sync()
    L, V, sig, info = (t.cpu().numpy() for t in (L, V, sig, info))
    assert np.all((info & 3) == 0), info
    Lo, Vo = OP.lift_pieces(X, piece_rows, Om, ell, w=w)
    Xd = X.astype(np.float64)
    xn = np.sqrt((Xd * Xd).sum(1))
    for q in range(pieces):
        r0, r1 = q * piece_rows, min(n, (q + 1) * piece_rows)
        sin = OR.projector_distance(V[q].astype(np.float64), Vo[q])
        assert sin <= 1e-4, (q, sin)
        err = np.sqrt(((L[r0:r1] - Lo[r0:r1]) ** 2).sum(1))
        assert np.all(err <= (sin + 1e-5) * xn[r0:r1]), (q, float((err / xn[r0:r1]).max()), sin)
        # Eckart-Young per piece: the residual of the GPU's lift against the full SVD's optimum
        wq = None if w is None else w[r0:r1]
        _, opt_sig = OR.exact_top(Xd[r0:r1], min(r1 - r0, d), w=wq)
        opt = float((opt_sig[ell:] ** 2).sum())
        res = OR.best_fit_error(Xd[r0:r1], V[q].astype(np.float64), w=wq)
        assert opt * (1 - 1e-6) <= res <= opt * (1 + 1e-3) + 1e-6 * float((opt_sig ** 2).sum())
        # each piece adds ell dimensions to the lifted point set
        assert OP.intrinsic_dimension(L[:r1].astype(np.float64), rel_tol=1e-4) == ell * (q + 1)


def test_piecy_lift_refuses_a_short_last_piece(gb):
    """Every piece needs at least s rows (the sketch has s columns): a ragged last piece of fewer
    rows is refused before anything is queued."""
    d, s = 64, 16
    X = T(np.zeros((1010, d), np.float32))
    Om = T(np.zeros((3, d, s), np.float32))
    with pytest.raises(gb.GbkmError) as e:
        gb.kmeans_piecy_lift(X, 500, Om, 8)
    assert e.value.code == gb.GBKM_EINVAL
