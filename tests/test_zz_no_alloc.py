"""The allocation-free update entry point against the regular one, through the C ABI.

kmeans_update_noalloc serves callers that cannot allocate device memory: it runs the
same update kernels on a fixed scratch block compiled into the library instead of a
context's workspace.  Both paths are deterministic and run the same kernels in the same
order of summation, so their results must be bitwise equal, call after call, although the
shared block keeps the previous call's contents.  The calls below cover both label-sorting
paths (k <= 2,048: shared-memory histograms; k > 2,048: a global histogram that the call
clears itself) and switch between them on the same block.  One result is also checked against
the FP64 oracle.  This file is named to be collected last, and works alone in a fresh process too.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import CENTROID_REL, COST_REL_F32, centroid_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _case(n, d, k, seed, weighted):
    X, z = synth.gaussian_mixture(n, d, min(k, 64), seed=seed)
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, max(1, k - 1), size=n).astype(np.int32) if k > 64 else (z % max(1, k - 1)).astype(np.int32)
    C_old = synth.gaussian_mixture(k, d, min(k, 64), seed=seed + 1)[0]   # cluster k-1 stays empty
    w = synth.integer_weights(n, seed=seed) if weighted else None
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return X, lab, t(X), t(lab), t(C_old), t(w)


def _check_same(a, b):
    """Bitwise equality of every output of the two entry points."""
    torch.cuda.synchronize()
    for key in ("C_new", "counts", "cost_old", "cost_new", "n_empty"):
        assert torch.equal(a[key], b[key]), f"{key} differs between kmeans_update_noalloc and kmeans_update"


def test_noalloc_update_matches_update_call_after_call(gb, orc):
    torch.cuda.set_device(0)
    # call 1: unweighted, aligned rows, shared-memory histograms (k <= 2,048)
    X, lab, Xg, lg, Cg, _ = _case(30_000, 128, 40, seed=21, weighted=False)
    ref = gb.kmeans_update(Xg, lg, Cg)
    got = gb.kmeans_update_noalloc(Xg, lg, Cg)
    _check_same(got, ref)
    # the same result against the FP64 oracle, within the update's tolerances
    o = orc.update(X, lab, Cg.cpu().numpy().astype(np.float64))
    assert np.array_equal(got["counts"].cpu().numpy(), o["N"])
    assert centroid_err(got["C_new"].cpu().numpy(), o["C_new"], X, lab) <= CENTROID_REL
    assert float(got["cost_new"].item()) == pytest.approx(o["cost_new"], rel=COST_REL_F32)
    # call 2, right after: a different, weighted, unaligned problem on the same scratch block
    _, _, Xg2, lg2, Cg2, wg2 = _case(7_001, 37, 13, seed=22, weighted=True)
    ref2 = gb.kmeans_update(Xg2, lg2, Cg2, w=wg2)
    _check_same(gb.kmeans_update_noalloc(Xg2, lg2, Cg2, w=wg2), ref2)
    # call 3: k > 2,048 takes the global-histogram path, whose table must be cleared by the call
    # although the block holds call 2's data
    _, _, Xg3, lg3, Cg3, _ = _case(20_000, 32, 3_000, seed=23, weighted=False)
    ref3 = gb.kmeans_update(Xg3, lg3, Cg3)
    _check_same(gb.kmeans_update_noalloc(Xg3, lg3, Cg3), ref3)
    _check_same(gb.kmeans_update_noalloc(Xg3, lg3, Cg3), ref3)
    # and the first problem again, after the large-k calls
    _check_same(gb.kmeans_update_noalloc(Xg, lg, Cg), ref)


def test_noalloc_update_rejects_problems_beyond_its_scratch(gb):
    """A problem whose scratch would exceed the fixed block is refused before anything is queued.
    With n = 20,000,000 the row permutation alone takes 4 n = 80 MB > 64 MiB, whatever the other
    terms; the size check precedes every launch, so the small buffers passed here are never read."""
    torch.cuda.set_device(0)
    n, d, k = 20_000_000, 16, 8
    assert 4 * n > gb.NOALLOC_SCRATCH_BYTES  # refused by the permutation term alone
    assert gb.kmeans_update_scratch_bytes(n, d, k) > gb.NOALLOC_SCRATCH_BYTES
    small = torch.empty(16, dtype=torch.float32, device=DEV)
    out = torch.empty(16, dtype=torch.float32, device=DEV)
    lab = torch.zeros(16, dtype=torch.int32, device=DEV)
    rc = gb.load().kmeans_update_noalloc(None, gb._ptr(small), n, d, None, gb._ptr(lab), k,
                                         gb._ptr(small), gb._ptr(out), None, None, None, None)
    assert rc == gb.GBKM_ETOOBIG
