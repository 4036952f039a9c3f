"""Randomised truncated SVD of a piece -- TEST INFRASTRUCTURE ONLY (FP64, numpy).

Section 2.2: a piece A (n points of dimension d, one point per row) is replaced by its projection
A_l = U D_l V^T onto the best-fit subspace of dimension l, spanned by the top l right singular
vectors V.  The paper computes them with a randomised truncated SVD after Halko, Martinsson and
Tropp (2011), as the redSVD library does: the columns of A are reduced by a random matrix, then
the rows, and only the small matrix left over is decomposed.  Section 2.3.2: for weighted points
the rows are scaled by sqrt(w_i) first; the best-fit subspace of that matrix is the one of the
matrix holding w_i copies of every row.  Section 3 (the redSVD comparison) measures a result by
||A - A_l'||_F^2 against the optimum ||A - A_l||_F^2 of the full SVD.

The steps below follow that order; numpy's QR and SVD serve as library steps.  The random matrix
is an input (the same one is handed to the CUDA path).  Pinned in tests/test_oracle_rsvd.py against
exact low-rank recovery, the Eckart-Young optimum of the full SVD, and the replicated-rows matrix
of Section 2.3.2.
"""
from __future__ import annotations

import numpy as np


def weighted(A, w=None):
    """A' = diag(sqrt(w)) A (Section 2.3.2); A itself when w is None."""
    A = np.asarray(A, dtype=np.float64)
    if w is None:
        return A
    return A * np.sqrt(np.asarray(w, dtype=np.float64))[:, None]


def rsvd(A, Omega, ell, w=None):
    """Top-ell right singular vectors (d x ell, columns) and singular values of A' by the randomised
    scheme: Y = A' Omega (columns reduced to s), Q an orthonormal basis of range(Y), B = Q^T A'
    (rows reduced to s), then the SVD of the s x d matrix B."""
    Ap = weighted(A, w)
    Om = np.asarray(Omega, dtype=np.float64)
    assert Om.shape[0] == Ap.shape[1] and ell <= Om.shape[1]
    Y = Ap @ Om
    Q, _ = np.linalg.qr(Y)
    B = Q.T @ Ap
    _, sig, Vt = np.linalg.svd(B, full_matrices=False)
    return Vt[:ell].T.copy(), sig[:ell].copy()


def exact_top(A, ell, w=None):
    """The full SVD's top-ell right singular vectors and singular values of A' (the paper's
    lapack++ baseline)."""
    _, sig, Vt = np.linalg.svd(weighted(A, w), full_matrices=False)
    return Vt[:ell].T.copy(), sig[:ell].copy()


def best_fit_error(A, V, w=None):
    """||A' - A' V V^T||_F^2: Section 3's error measure for a basis V with orthonormal columns."""
    Ap = weighted(A, w)
    V = np.asarray(V, dtype=np.float64)
    R = Ap - (Ap @ V) @ V.T
    return float((R * R).sum())


def projector_distance(V1, V2):
    """Spectral norm of V1 V1^T - V2 V2^T (the sine of the largest principal angle)."""
    V1 = np.asarray(V1, dtype=np.float64)
    V2 = np.asarray(V2, dtype=np.float64)
    return float(np.linalg.norm(V1 @ V1.T - V2 @ V2.T, 2))


def sign_normalised(V):
    """Columns flipped so that the entry of largest magnitude (lowest row on ties) is positive."""
    V = np.array(V, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V
