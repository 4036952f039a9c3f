"""Tolerances and comparisons shared by the GPU parity tests.

Tolerances (stated by the workload definition, or derived from the arithmetic):
  labels    bit-identical to the FP64 oracle except rows whose oracle top-2 gap
            (d2 - d1) / d1 is below 1e-5 (certified near-ties);
  centroids ||c - c*||_2 / max(||c*||_2, rms radius of the cluster) <= 1e-5;
  cost      relative 1e-6 for the FP32 path, 1e-4 for BF16 / FP8 forms.
"""
import numpy as np

TIE_REL = 1e-5
CENTROID_REL = 1e-5
COST_REL_F32 = 1e-6
COST_REL_LOWP = 1e-4


def oracle_gap(orc, X, d1, d2):
    return orc.near_tie_gap(X, d1, d2)


def assert_labels_match(orc, X, C, labels_gpu, tie_rel=TIE_REL):
    """Labels equal the oracle's exact nearest center except on certified near-ties; on those
    the GPU's choice must still be one of the tied centers (its distance within the band)."""
    lab, d1, d2 = orc.assign(X, C)
    labels_gpu = np.asarray(labels_gpu)
    gap = orc.near_tie_gap(X, d1, d2)
    diff = labels_gpu != lab
    bad = diff & (gap >= tie_rel)
    assert not bad.any(), (f"{int(bad.sum())} labels differ outside the near-tie band; "
                           f"first rows {np.nonzero(bad)[0][:5]}")
    if diff.any():
        Xd = np.asarray(X, np.float64)
        rows = np.nonzero(diff)[0]
        dg = ((Xd[rows] - np.asarray(C, np.float64)[labels_gpu[rows]]) ** 2).sum(1)
        assert np.all(dg <= d1[rows] * (1 + 2 * tie_rel) + 1e-30)
    return lab, d1, d2, int(diff.sum())


def centroid_err(C_gpu, C_ref, X, labels):
    """max over clusters of ||c - c*|| / max(||c*||, rms radius of the cluster)."""
    C_gpu = np.asarray(C_gpu, np.float64)
    C_ref = np.asarray(C_ref, np.float64)
    Xd = np.asarray(X, np.float64)
    worst = 0.0
    for j in range(C_ref.shape[0]):
        m = labels == j
        rad = np.sqrt(((Xd[m] - C_ref[j]) ** 2).sum(1).mean()) if m.any() else 0.0
        den = max(np.linalg.norm(C_ref[j]), rad, 1e-30)
        worst = max(worst, np.linalg.norm(C_gpu[j] - C_ref[j]) / den)
    return worst
