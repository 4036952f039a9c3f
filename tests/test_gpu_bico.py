"""GPU parity of the batched weighted nearest-reference query (Section 2.1 clustering features,
Section 2.3.1 weighted insertion) against oracle/bico.py, through the C ABI.

The reference search is the exact assignment step (labels equal the FP64 full scan except on
certified near-ties, where either tied reference is accepted and the rest is recomputed for the
GPU's choice).  The squared distance to the feature's centroid is FP64 on both sides from the same
centroid bits (mu = S / N rounded once), so it agrees to the summation order: (d + 2) 2^-53
relative.  The insertable count is an integer decided in FP64 by the same rule on both sides and
must be equal; with continuous random data no quotient lands within rounding of an integer.
"""
import numpy as np
import pytest
import torch

from oracle import bico as OB
from paper_1502_04265_gb300 import synth
from parity_util import assert_labels_match

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T_(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _snapshot(refs, seed):
    P, f = synth.bico_members(refs, seed)
    m, d = refs.shape
    N, S, Q = np.zeros(m), np.zeros((m, d)), np.zeros(m)
    for j in range(m):
        N[j], S[j], Q[j] = OB.cf_of(P[f == j])
    return N, S, Q


@pytest.mark.parametrize("n,d,m,form", [(5000, 64, 300, "f32"), (3001, 128, 1000, "f32"), (4000, 256, 500, "bf16"),
                                        (700, 40, 17, "f32")])
def test_bico_query_matches_oracle(gb, orc, n, d, m, form):
    refs, _ = synth.gaussian_mixture(m, d, max(2, m // 4), seed=m + d)
    N, S, Q = _snapshot(refs, seed=d)
    cerr = np.array([OB.cf_error(N[j], S[j], Q[j]) for j in range(m)])
    T = float(np.quantile(cerr, 0.8))          # a fifth of the features are already over T
    X = synth.bico_batch(refs, n, seed=n)
    w = synth.integer_weights(n, seed=n, max_w=20)
    Xg = T_(X)
    Xop, Xr = gb.kmeans_quantize(Xg, "bf16") if form == "bf16" else (None, None)
    ref, d2, take = gb.kmeans_bico_query(Xg, T_(refs), T_(N), T_(S), T_(Q), T, w=T_(w), Xop=Xop, Xop_scales=Xr,
                                         compute=form)
    gb.gbkm_sync()
    ref, d2, take = ref.cpu().numpy(), d2.cpu().numpy(), take.cpu().numpy()
    j_or, d2_or, take_or = OB.batch_query(X, w, refs, N, S, Q, T)
    assert_labels_match(orc, X, refs.astype(np.float64), ref)
    same = ref == j_or
    # the rows whose nearest reference is a certified near-tie: the oracle's rule for the GPU's choice
    for i in np.nonzero(~same)[0]:
        f = int(ref[i])
        mu = S[f] / N[f]
        d2_or[i] = float((X[i].astype(np.float64) - mu) @ (X[i].astype(np.float64) - mu))
        take_or[i] = OB.insertable(N[f], cerr[f], T, d2_or[i], float(w[i]))
    np.testing.assert_allclose(d2, d2_or, rtol=(d + 2) * 2.0 ** -53 * 4, atol=0)
    assert np.array_equal(take, take_or), f"{int((take != take_or).sum())} counts differ"
    # all three branches of the rule occur
    assert (take == w).sum() >= 10, "no point fits whole"
    assert ((take > 0) & (take < w)).sum() >= 10, "no point fits in part"
    assert (take == 0).sum() >= 10, "no point is refused"
    over = cerr[ref] > T
    assert np.all(take[over] == 0)


def test_bico_query_unweighted_and_threshold_zero(gb):
    """w = NULL means one copy per point; T = 0 admits a point only where it leaves the error at 0:
    a point on the centroid of a one-point feature."""
    d, m = 16, 8
    refs = np.arange(m * d, dtype=np.float32).reshape(m, d)
    N = np.ones(m)
    S = refs.astype(np.float64)
    Q = (S * S).sum(1)
    X = np.concatenate([refs[3:4], refs[5:6] + np.float32(0.5)])
    ref, d2, take = gb.kmeans_bico_query(T_(X), T_(refs), T_(N), T_(S), T_(Q), 0.0)
    gb.gbkm_sync()
    assert ref.cpu().tolist() == [3, 5]
    assert d2.cpu().tolist() == [0.0, 0.25 * d]
    assert take.cpu().tolist() == [1.0, 0.0]
