"""Weighted insertion into BICO's clustering features -- TEST INFRASTRUCTURE ONLY (FP64, numpy).

Section 2.1: a clustering feature (CF) of a point set holds its size, the sum of its points and the
sum of their squared lengths, which fixes the cost of the set against any one center.  Section 2.3.1
(weighted BICO): a weighted point (x, w) stands for w copies of x.  The nearest reference point is
found once for all copies.  Adding w copies to a feature with s points, centroid mu and error c
raises the error by s w / (s + w) ||x - mu||^2, so at most w' copies fit under the threshold T:
all w when s ||x - mu||^2 - T + c <= 0, else min(w, (sT - sc) / (s ||x - mu||^2 - T + c)).

The batched query below answers, for every point of a batch and one fixed snapshot of the
features, which reference is nearest and how many copies that feature can take; the sequential
tree that applies the answers stays out of it.  Pinned in tests/test_oracle_bico.py against the
direct definition of a feature's error and the threshold inequality.
"""
from __future__ import annotations

import math

import numpy as np


def cf_of(P, w=None):
    """Clustering feature (N, S, Q) of the rows of P with weights w: N = sum w, S = sum w x,
    Q = sum w ||x||^2."""
    P = np.asarray(P, dtype=np.float64)
    w = np.ones(P.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    return float(w.sum()), (P * w[:, None]).sum(axis=0), float((w * (P * P).sum(axis=1)).sum())


def cf_error(N, S, Q):
    """The feature's error sum w ||x - mu||^2 = Q - ||S||^2 / N (0 for an empty feature)."""
    if N <= 0:
        return 0.0
    S = np.asarray(S, dtype=np.float64)
    return float(Q - S @ S / N)


def error_increase(s, mu, x, w):
    """Rise of the error when w copies of x join a feature of s points with centroid mu:
    s w / (s + w) ||x - mu||^2 (Section 2.3.1)."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(mu, dtype=np.float64)
    return s * w / (s + w) * float(d @ d)


def insertable(s, c, T, d2, w):
    """Copies of a point at squared distance d2 from the centroid that a feature (s points, error
    c) takes before its error exceeds T: all w when s d2 - T + c <= 0, else
    min(w, (sT - sc) / (s d2 - T + c)) rounded down to whole copies (weights are integral), and
    none when the feature's error already exceeds T (the paper leaves c > T open)."""
    den = s * d2 - T + c
    if den <= 0:
        return float(w)
    return float(max(0, min(w, math.floor((s * T - s * c) / den))))


def nearest_reference(X, refs):
    """Index of the nearest reference row (lowest index on ties) and the squared distance, FP64."""
    X = np.asarray(X, dtype=np.float64)
    R = np.asarray(refs, dtype=np.float64)
    D = ((X[:, None, :] - R[None, :, :]) ** 2).sum(axis=2)
    j = np.argmin(D, axis=1)
    return j.astype(np.int32), D[np.arange(X.shape[0]), j]


def batch_query(X, w, refs, N, S, Q, T):
    """For every point of a batch: its nearest reference j (the reference points are the features'
    own reference rows), the squared distance to feature j's centroid, and the copies w' of the
    point that feature j takes under threshold T, all against the given snapshot (N, S, Q)."""
    X = np.asarray(X, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    j, _ = nearest_reference(X, refs)
    d2 = np.empty(X.shape[0])
    take = np.empty(X.shape[0])
    for i in range(X.shape[0]):
        f = j[i]
        mu = S[f] / N[f]
        diff = X[i] - mu
        d2[i] = float(diff @ diff)
        take[i] = insertable(N[f], cf_error(N[f], S[f], Q[f]), T, d2[i], w[i])
    return j, d2, take
