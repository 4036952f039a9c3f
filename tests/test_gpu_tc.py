"""GPU parity of the tcgen05 engine (distance GEMM + fused top-2 epilogue, projection GEMM).

Every precision form must give the exact nearest center (bit-identical to the FP64 oracle
outside the 1e-5 near-tie band) because rows inside the certified error band are re-resolved
exactly; the expanded-form min distance carries the form's rounding.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import assert_labels_match

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _data(n, d, k, seed):
    X, _ = synth.gaussian_mixture(n, d, max(2, k // 2), seed=seed)
    C = synth.gaussian_mixture(k, d, max(2, k // 2), seed=seed + 1)[0]
    return X, C


def _assign(gb, X, C, form, **kw):
    Xg, Cg = T(X), T(C)
    Xop, sc = None, None
    if form in ("bf16", "fp8"):
        Xop, sc = gb.kmeans_quantize(Xg, form)
    n = X.shape[0]
    md = torch.empty(n, dtype=torch.float32, device=DEV)
    nre = torch.zeros(1, dtype=torch.int64, device=DEV)
    lab = gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=sc, compute=form, engine="tcgen05",
                           min_d2=md, n_rechecked=nre, **kw)
    gb.gbkm_sync()
    return H(lab), H(md), int(H(nre)[0])


def test_tc_smallest_tile_bf16(gb, orc):
    """One 128-row tile, one K block, one 16-wide center chunk: the smallest tcgen05 case."""
    X, C = _data(128, 64, 16, seed=1)
    lab, md, nre = _assign(gb, X, C, "bf16")
    assert_labels_match(orc, X, C.astype(np.float64), lab)


TC_CASES = [
    (1000, 64, 10),      # ragged last tile, one K block, k padded 10 -> 16
    (3000, 1024, 100),   # the high-dimensional shape, scaled down in n
    (2100, 72, 300),     # two center chunks; K tail (72 = 64 + 8 -> OOB zero fill)
    (700, 128, 1000),    # four center chunks
    (257, 256, 1),       # k = 1
]


@pytest.mark.parametrize("form", ["bf16", "f32", "bf16x2"])
@pytest.mark.parametrize("n,d,k", TC_CASES)
def test_tc_assign_exact_labels(gb, orc, form, n, d, k):
    X, C = _data(n, d, k, seed=n + d + k)
    if form == "bf16x2":
        lab, md, nre = _assign(gb, X, C, "bf16", center_terms=2)
    else:
        lab, md, nre = _assign(gb, X, C, form)
    ref, d1, d2, _ = assert_labels_match(orc, X, C.astype(np.float64), lab)
    xn = orc.row_norms(X)
    cn = (C.astype(np.float64) ** 2).sum(1).max()
    rel = 1e-4 if form == "f32" else 2.0 ** -6
    assert np.all(np.abs(md - d1) <= rel * np.sqrt(xn * cn) * 2 + 1e-3)


@pytest.mark.parametrize("n,d,k", [(1500, 64, 40), (900, 128, 257), (640, 48, 9)])
def test_tc_assign_fp8_exact_labels(gb, orc, n, d, k):
    X, C = _data(n, d, k, seed=3 * n + k)
    lab, md, nre = _assign(gb, X, C, "fp8")
    assert_labels_match(orc, X, C.astype(np.float64), lab)


def test_tc_matches_simt_engine(gb):
    X, C = _data(5000, 256, 77, seed=9)
    Xg, Cg = T(X), T(C)
    a = H(gb.kmeans_assign(Xg, Cg, engine="simt"))
    b = H(gb.kmeans_assign(Xg, Cg, compute="f32", engine="tcgen05"))
    Xb, _ = gb.kmeans_quantize(Xg, "bf16")
    c = H(gb.kmeans_assign(Xg, Cg, Xop=Xb, compute="bf16", engine="tcgen05"))
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_tc_planted_ties(gb, orc):
    rng = np.random.default_rng(5)
    d, k = 64, 16
    C = rng.integers(-8, 8, size=(k, d)).astype(np.float32) * 2.0
    C[7] = C[3]
    X = np.concatenate([0.5 * (C[0:1] + C[1:2]), 0.5 * (C[2:3] + C[5:6]), C[3:4] + 0.25,
                        rng.normal(size=(300, d)).astype(np.float32) * 6]).astype(np.float32)
    for form in ("bf16", "f32"):
        lab, _, nre = _assign(gb, X, C, form)
        ref, _, _ = orc.assign(X, C.astype(np.float64))
        assert np.array_equal(lab[:3], ref[:3]) and lab[2] == 3
        assert nre >= 3
        assert_labels_match(orc, X, C.astype(np.float64), lab)


def _tf32(a):
    """The top 19 bits of every FP32 value (what one TF32 term keeps)."""
    a = np.ascontiguousarray(a, np.float32)
    return (a.view(np.uint32) & np.uint32(0xffffe000)).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("xt", ["f32", "bf16"])
@pytest.mark.parametrize("n,d,r", [(1000, 256, 64), (300, 2048, 64), (129, 64, 16), (200, 512, 256)])
def test_tc_project_and_lift(gb, orc, xt, n, d, r):
    """Y = X V on the tensor cores (BF16, or FP32 X in the 3xTF32 form) and the lift Y V^T (3xTF32).

    Worst-case bounds per element: BF16 |Y - Yr| <= (2u + d 2^-22) ||x|| (u = 2^-8, ||v_q|| = 1);
    3xTF32 (3.01 2^-20 + 3d 2^-22) ||x||.  The FP32 form must also beat a single TF32 term: its error
    is at most half the error that truncating X and V to TF32 gives on the same data (computed here
    in FP64).  The lift is compared with the FP64 lift of the GPU's own Y, so that only its own
    rounding counts, and must likewise beat a single TF32 term by 2x."""
    Q = synth.orthonormal_basis(d, min(r, 8), seed=d)
    X, _ = synth.subspace_mixture_chunk(Q, 0, n, 10, seed=r)
    V = synth.orthonormal_basis(d, r, seed=r + 1).astype(np.float32)
    Xg = T(X)
    Xin = Xg if xt == "f32" else gb.kmeans_quantize(Xg, "bf16")[0]
    Y, L = gb.kmeans_project_block(Xin, T(V), lift=True)
    Y, L = H(Y), H(L)
    V64 = V.astype(np.float64)
    Yr = orc.project(X, V64)
    xn = np.sqrt(orc.row_norms(X))[:, None]
    if xt == "bf16":
        u = 2.0 ** -8
        assert np.all(np.abs(Y - Yr) <= (2 * u + d * 2.0 ** -22) * xn + 1e-5)
    else:
        assert np.all(np.abs(Y - Yr) <= (3.01 * 2.0 ** -20 + 3 * d * 2.0 ** -22) * xn + 1e-6)
        single = np.abs(_tf32(X) @ _tf32(V) - Yr).max()
        assert np.abs(Y - Yr).max() <= 0.5 * single
    Lg = Y.astype(np.float64) @ V64.T           # the exact lift of the GPU's Y
    yn = np.sqrt((Y.astype(np.float64) ** 2).sum(1))[:, None]
    assert np.all(np.abs(L - Lg) <= (3.01 * 2.0 ** -20 + 3 * r * 2.0 ** -22) * yn + 1e-6)
    single = np.abs(_tf32(Y) @ _tf32(V).T - Lg).max()
    assert np.abs(L - Lg).max() <= 0.5 * single


@pytest.mark.parametrize("form", ["bf16", "f32", "fp8"])
def test_tc_band_across_chunks_and_overflow(gb, orc, form):
    """Near-tie bands whose members sit in different 256-center chunks, and a band larger than the
    candidate list (12 identical centers, so the recheck scans every center): exact labels."""
    rng = np.random.default_rng(11)
    d, k = 64, 1000
    C = rng.uniform(-10, 10, size=(k, d)).astype(np.float32)
    C[700] = C[3] + np.float32(1e-3)
    C[999] = C[3] - np.float32(1e-3)
    C[900:912] = C[500]
    X = np.concatenate([C[3] + rng.normal(size=(200, d)).astype(np.float32) * 0.5,
                        C[500] + rng.normal(size=(200, d)).astype(np.float32) * 0.5,
                        rng.uniform(-10, 10, size=(300, d)).astype(np.float32)]).astype(np.float32)
    lab, _, nre = _assign(gb, X, C, form)
    assert nre >= 400
    assert_labels_match(orc, X, C.astype(np.float64), lab)
    # the 12 identical centers tie exactly: the lowest index wins
    assert np.all(lab[200:400] == 500)


@pytest.mark.parametrize("terms", [1, 2])
@pytest.mark.parametrize("scale", [3.0, 10.0])
def test_tc_bf16_pairs_near_bisectors(gb, orc, scale, terms):
    """Pairs of close centers far from the origin and points scattered around each pair's
    midpoint: many points sit near a bisector, where the BF16 rounding decides, and both BF16
    forms' bounds (the two-term centers' one grows with the distances) must flag every point
    they cannot certify."""
    rng = np.random.default_rng(int(scale))
    d, pairs, n = 256, 32, 20000
    mu = rng.uniform(-scale, scale, size=(pairs, d))
    delta = rng.normal(size=(pairs, d)) * (5.0 / np.sqrt(d))
    C = np.concatenate([mu + delta, mu - delta]).astype(np.float32)
    z = rng.integers(0, pairs, size=n)
    X = (mu[z] + rng.normal(size=(n, d)) * 0.3).astype(np.float32)
    lab, _, nre = _assign(gb, X, C, "bf16", center_terms=terms)
    assert_labels_match(orc, X, C.astype(np.float64), lab)
    assert nre > 0 and (scale > 5 or terms == 1 or nre < n)


def test_bf16_residual_band_exact_with_fewer_rechecks(gb, orc):
    """The band built from the rows' and centers' actual BF16 residuals (side data of the quantised
    copy) is narrower than the worst case u ||x|| ||c||: fewer rows are rechecked, and the labels
    are still the exact nearest centers."""
    X, _ = synth.gaussian_mixture(6000, 1024, 100, seed=21)
    C = X[(synth.seed_uniforms(100, 3) * 6000).astype(np.int64)].copy()
    Xg, Cg = T(X), T(C)
    Xb, Xr = gb.kmeans_quantize(Xg, "bf16")
    out = []
    for sc in (None, Xr):
        nre = torch.zeros(1, dtype=torch.int64, device=DEV)
        lab = gb.kmeans_assign(Xg, Cg, Xop=Xb, Xop_scales=sc, compute="bf16", engine="tcgen05", n_rechecked=nre)
        gb.gbkm_sync()
        assert_labels_match(orc, X, C.astype(np.float64), H(lab))
        out.append(int(H(nre)[0]))
    worst, resid = out
    assert resid <= worst
    if worst >= 100:
        assert resid < worst
