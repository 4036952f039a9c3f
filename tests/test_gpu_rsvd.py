"""GPU parity of the randomised truncated SVD (Section 2.2; weighted rows, Section 2.3.2) against the
FP64 oracle given the same random matrix.

Tolerances.  The passes over A run in FP32 (sums of d or n products: relative errors of order
1e-6 for these sizes), the Gram matrices in double-float, the Cholesky factors in FP64 and the
small one-sided Jacobi in FP32 (convergence threshold s * 1.2e-7).  Singular values therefore
agree to 1e-4 of the largest, the basis to 1e-3 per entry where consecutive singular values are
at least 5% apart, and the error measure of Section 3 to 1e-4 relative.
"""
import numpy as np
import pytest
import torch

from oracle import rsvd as R
from paper_1502_04265_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _run(gb, A, Om, ell, w=None):
    V, s, info = gb.kmeans_rsvd(T(A), T(Om), ell, w=None if w is None else T(w))
    torch.cuda.synchronize()
    return V.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64), int(info.cpu().numpy()[0])


def _check(A, Om, ell, V, s, w=None, v_tol=1e-3, gap=0.05):
    A32 = np.asarray(A, np.float32).astype(np.float64)
    Vo, so = R.rsvd(A32, Om.astype(np.float64), ell, w=w)
    Vo = R.sign_normalised(Vo)
    assert np.max(np.abs(s - so)) <= 1e-4 * so[0]
    assert np.max(np.abs(V.T @ V - np.eye(ell))) <= 1e-4
    # columns whose singular value is separated from both neighbours by the gap
    rel = np.abs(np.diff(so)) / so[:-1]
    sep = [j for j in range(ell) if (j == 0 or rel[j - 1] >= gap) and (j == ell - 1 or rel[j] >= gap)]
    if sep:
        assert np.max(np.abs(V[:, sep] - Vo[:, sep])) <= v_tol
    e, eo = R.best_fit_error(A32, V, w), R.best_fit_error(A32, Vo, w)
    assert e == pytest.approx(eo, rel=1e-4)
    return Vo, so


def _low_rank(n, d, r, top, seed, noise):
    sig = np.geomspace(top, top / 100.0, r)
    A = synth.planted_spectrum(n, d, sig, seed=seed)
    A += noise * np.random.default_rng(seed).standard_normal((n, d))
    return A.astype(np.float32)


# s spans the Gram kernel's three tilings (up to 88, 96-124 and 128 columns)
@pytest.mark.parametrize("n,d,r,s,ell", [(3000, 300, 40, 48, 32), (1000, 203, 30, 32, 5), (257, 64, 20, 16, 16),
                                         (5000, 512, 100, 128, 100), (2400, 256, 70, 96, 64),
                                         (1700, 320, 90, 112, 80)])
def test_rsvd_matches_oracle(gb, n, d, r, s, ell):
    A = _low_rank(n, d, r, 100.0, seed=n + d, noise=1e-3)
    Om = synth.gaussian_sketch(d, s, seed=s)
    V, sg, info = _run(gb, A, Om, ell)
    _check(A, Om, ell, V, sg)


def test_rsvd_weighted_matches_oracle(gb):
    A = _low_rank(2000, 160, 30, 50.0, seed=3, noise=1e-3)
    w = synth.integer_weights(2000, seed=4, max_w=5).astype(np.float32)
    Om = synth.gaussian_sketch(160, 32, seed=5)
    V, sg, _ = _run(gb, A, Om, 20, w=w)
    _check(A, Om, 20, V, sg, w=w.astype(np.float64))
    V0, _, _ = _run(gb, A, Om, 20)
    assert R.projector_distance(V, V0) > 1e-3   # the weights change the subspace


def test_rsvd_rank_deficient_recovers_exact_subspace(gb):
    """rank 10 < s = 32: the planted singular values and vectors come back; the clamped pivots
    of the rank-deficient Gram matrices are reported in info bit 0 or absorbed by the shift."""
    sig = np.geomspace(30.0, 3.0, 10)
    A = synth.planted_spectrum(1500, 120, sig, seed=9).astype(np.float32)
    W = synth.orthonormal_basis(120, 10, 20)
    Om = synth.gaussian_sketch(120, 32, seed=11)
    V, sg, info = _run(gb, A, Om, 8)
    np.testing.assert_allclose(sg, sig[:8], rtol=1e-4)
    assert R.projector_distance(V, W[:, :8]) < 1e-3
    assert 1 <= info >> 8 <= 30   # bits 8-15: the Jacobi sweeps run


def test_rsvd_stream_piece_recovers_planted_basis(gb):
    """A piece of the rank-64-subspace workload (d = 2,048, noise 0.1): s = 80, l = 64 matches the
    oracle and spans the planted subspace up to the noise."""
    Qp = synth.orthonormal_basis(2048, 64, 0)
    A, _ = synth.subspace_mixture_chunk(Qp, 0, 16384, 500, 0)
    Om = synth.gaussian_sketch(2048, 80, seed=1)
    V, sg, info = _run(gb, A, Om, 64)
    assert (info & 0xFF) == 0
    _check(A, Om, 64, V, sg)
    assert R.projector_distance(V, Qp) < 0.1


def test_rsvd_rejects_bad_shapes(gb):
    A = torch.zeros((100, 40), dtype=torch.float32, device=DEV)
    for s, ell in ((24, 8), (32, 40), (48, 8), (144, 8)):
        Om = torch.zeros((40, s), dtype=torch.float32, device=DEV)
        with pytest.raises(gb.GbkmError) as e:
            gb.kmeans_rsvd(A, Om, ell)
        assert e.value.code == gb.GBKM_EINVAL
