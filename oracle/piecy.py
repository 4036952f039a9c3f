"""Per-piece bases with the d-dimensional lift -- TEST INFRASTRUCTURE ONLY (FP64, numpy).

Section 2.2 (piecy): the input is read in pieces of p points; each piece is replaced by its
projection onto its own best-fit subspace of dimension l, A_l = A V V^T, which keeps d coordinates
but has intrinsic dimension l, and the projected points go on to the clustering.  Every piece adds
up to l dimensions to the point set as a whole (Section 2.3, piecy-mr), which is what the
intrinsic-dimension check below measures.  The basis of each piece comes from the randomised SVD
of oracle.rsvd with that piece's random matrix.  Pinned in tests/test_oracle_piecy.py.
"""
from __future__ import annotations

import numpy as np

from . import rsvd as _rsvd


def lift_pieces(X, piece_rows, Omegas, ell, w=None):
    """Pieces of `piece_rows` consecutive rows (the last may be shorter), each projected onto the
    span of its own top-ell basis: returns the lifted n x d matrix and the list of bases."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    out = np.empty_like(X)
    bases = []
    for q, r0 in enumerate(range(0, n, piece_rows)):
        r1 = min(n, r0 + piece_rows)
        wq = None if w is None else np.asarray(w, dtype=np.float64)[r0:r1]
        V, _ = _rsvd.rsvd(X[r0:r1], Omegas[q], ell, w=wq)
        out[r0:r1] = (X[r0:r1] @ V) @ V.T
        bases.append(V)
    return out, bases


def intrinsic_dimension(Y, rel_tol=1e-9):
    """Numerical rank of Y: singular values above rel_tol times the largest."""
    sv = np.linalg.svd(np.asarray(Y, dtype=np.float64), compute_uv=False)
    return int((sv > rel_tol * sv[0]).sum()) if sv.size and sv[0] > 0 else 0
