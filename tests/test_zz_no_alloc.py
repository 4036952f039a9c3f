"""The allocation-free update entry point against the regular one, through the C ABI.

kmeans_update_noalloc serves callers that cannot allocate device memory: it runs the
same update kernels on a fixed scratch block compiled into the library instead of a
context's workspace.  Its results must equal kmeans_update's (same kernels, same order of
summation) on consecutive calls, since the shared block keeps the previous call's contents.
This file is named to be collected last, and works alone in a fresh process too.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import CENTROID_REL, COST_REL_F32, centroid_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _case(n, d, k, seed, weighted):
    X, z = synth.gaussian_mixture(n, d, k, seed=seed)
    lab = (z % max(1, k - 1)).astype(np.int32)   # one cluster left empty
    C_old = synth.gaussian_mixture(k, d, k, seed=seed + 1)[0]
    w = synth.integer_weights(n, seed=seed) if weighted else None
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return X, lab, t(X), t(lab), t(C_old), t(w)


def _check_same(gb, a, b, X, lab):
    torch.cuda.synchronize()
    assert np.array_equal(a["counts"].cpu().numpy(), b["counts"].cpu().numpy())
    assert int(a["n_empty"].item()) == int(b["n_empty"].item())
    ca, cb = a["C_new"].cpu().numpy(), b["C_new"].cpu().numpy()
    assert centroid_err(ca, cb.astype(np.float64), X, lab) <= CENTROID_REL
    for key in ("cost_old", "cost_new"):
        assert float(a[key].item()) == pytest.approx(float(b[key].item()), rel=COST_REL_F32)


def test_noalloc_update_matches_update_on_two_calls(gb):
    torch.cuda.set_device(0)
    # call 1: unweighted, aligned rows
    X, lab, Xg, lg, Cg, _ = _case(30_000, 128, 40, seed=21, weighted=False)
    ref = gb.kmeans_update(Xg, lg, Cg)
    got = gb.kmeans_update_noalloc(Xg, lg, Cg)
    _check_same(gb, got, ref, X, lab)
    # call 2, right after: a different, weighted, unaligned problem on the same scratch block
    X2, lab2, Xg2, lg2, Cg2, wg2 = _case(7_001, 37, 13, seed=22, weighted=True)
    ref2 = gb.kmeans_update(Xg2, lg2, Cg2, w=wg2)
    got2 = gb.kmeans_update_noalloc(Xg2, lg2, Cg2, w=wg2)
    _check_same(gb, got2, ref2, X2, lab2)
    # and the first problem again, whose stale scratch contents must not leak into the result
    got3 = gb.kmeans_update_noalloc(Xg, lg, Cg)
    _check_same(gb, got3, ref, X, lab)


def test_noalloc_update_rejects_problems_beyond_its_scratch(gb):
    """A problem whose scratch would exceed the fixed block is refused before anything is queued.
    With n = 20,000,000 the row permutation alone takes 4 n = 80 MB > 64 MiB, whatever the other
    terms; the size check precedes every launch, so the small buffers passed here are never read."""
    torch.cuda.set_device(0)
    n, d, k = 20_000_000, 16, 8
    assert 4 * n > gb.NOALLOC_SCRATCH_BYTES  # refused by the permutation term alone
    small = torch.empty(16, dtype=torch.float32, device=DEV)
    out = torch.empty(16, dtype=torch.float32, device=DEV)
    lab = torch.zeros(16, dtype=torch.int32, device=DEV)
    rc = gb.load().kmeans_update_noalloc(None, gb._ptr(small), n, d, None, gb._ptr(lab), k,
                                         gb._ptr(small), gb._ptr(out), None, None, None, None)
    assert rc == gb.GBKM_ETOOBIG
