"""Exact k-means optimum of tiny inputs by enumeration -- TEST INFRASTRUCTURE ONLY.

The k-means problem (Section 1) asks for the partition into at most k sets
minimising the summed squared distances to each set's centroid (Section 2:
mu(P) = sum x / |P| is the optimal center of a set).  For n <= 10 and k <= 3
all k^n labelings (at most 59,049) are enumerated in FP64; that gives the
optimum directly, with no heuristic involved.
"""
from __future__ import annotations

import itertools

import numpy as np


def partition_cost(X: np.ndarray, labels, k: int) -> float:
    """sum over sets of sum_{x in P} ||x - mu(P)||^2, FP64, empty sets cost nothing."""
    X = np.asarray(X, np.float64)
    total = 0.0
    for j in range(k):
        P = X[np.asarray(labels) == j]
        if len(P) == 0:
            continue
        mu = P.sum(axis=0) / len(P)
        total += float(((P - mu) ** 2).sum())
    return total


def optimum(X: np.ndarray, k: int):
    """(optimal cost, one optimal labeling, its centroids) by enumerating k^n labelings."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    if n > 10 or k > 3:
        raise ValueError("brute force is limited to n <= 10 and k <= 3")
    best, best_lab = np.inf, None
    for lab in itertools.product(range(k), repeat=n):
        if lab[0] != 0:  # labels are symmetric under renaming: fix the first point's set
            continue
        c = partition_cost(X, lab, k)
        if c < best:
            best, best_lab = c, np.array(lab, np.int32)
    cents = np.zeros((k, X.shape[1]))
    for j in range(k):
        P = X[best_lab == j]
        cents[j] = P.mean(axis=0) if len(P) else np.nan
    return best, best_lab, cents
