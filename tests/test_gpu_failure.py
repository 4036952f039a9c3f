"""Failure detection without a GPU fault (no trap, no bad address, no endless loop).

A bounded device wait that runs out: with gbkm_debug_stall_loads the tensor-core kernel's producer
issues no copy, so the issuer's first wait (for a copy that is never made) can only end by its
limit, set short here.  The launch must then drain, free its tensor memory and return; the next
gbkm_sync must report GBKM_ETIMEOUT (and clear it), and the same context must then give the exact
labels again.  A failed workspace allocation: gbkm_debug_fail_alloc makes the next workspace growth
fail as a failed cudaMalloc would; the call returns GBKM_ENOMEM before queuing anything, and the
next call on the context succeeds.
"""
import numpy as np
import pytest
import torch

from paper_1502_04265_gb300 import synth
from parity_util import CENTROID_REL, assert_labels_match, centroid_err

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _data(n, d, k, seed):
    X, _ = synth.gaussian_mixture(n, d, k, seed=seed)
    C = X[(synth.seed_uniforms(k, seed) * n).astype(np.int64)].copy()
    return X, C


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_bounded_wait_runs_out_and_the_context_recovers(gb, orc, form):
    X, C = _data(20_000, 256, 40, seed=5)
    Xg, Cg = torch.from_numpy(X).to(DEV), torch.from_numpy(C).to(DEV)
    ctx = gb.Context(0)
    Xop, Xr = gb.kmeans_quantize(Xg, "bf16", ctx=ctx) if form == "bf16" else (None, None)
    ref = gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=Xr, compute=form, engine="tcgen05", ctx=ctx)
    ctx.sync()
    ctx.set_wait_limit(1_000_000)            # 1 ms
    ctx.stall_loads(True)
    lab = torch.full((X.shape[0],), -7, dtype=torch.int32, device=DEV)
    gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=Xr, compute=form, engine="tcgen05", labels=lab, ctx=ctx)
    with pytest.raises(gb.GbkmError) as e:
        ctx.sync()
    assert e.value.code == gb.GBKM_ETIMEOUT
    torch.cuda.synchronize()                 # no CUDA error is left behind
    # the status word was cleared; back to normal operation on the same context
    ctx.stall_loads(False)
    ctx.set_wait_limit(0)
    ctx.sync()
    again = gb.kmeans_assign(Xg, Cg, Xop=Xop, Xop_scales=Xr, compute=form, engine="tcgen05", labels=lab, ctx=ctx)
    ctx.sync()
    assert torch.equal(again, ref)
    assert_labels_match(orc, X, C.astype(np.float64), again.cpu().numpy())
    ctx.close()


def test_failed_workspace_allocation_reports_enomem(gb, orc):
    X, C = _data(5_000, 64, 12, seed=6)
    Xg, Cg = torch.from_numpy(X).to(DEV), torch.from_numpy(C).to(DEV)
    lab = torch.from_numpy(orc.assign(X, C.astype(np.float64))[0]).to(DEV)
    ctx = gb.Context(0)                      # a fresh context: its workspace must grow first
    ctx.fail_next_allocs(1)
    C_new = torch.full_like(Cg, -1.0)
    with pytest.raises(gb.GbkmError) as e:
        gb.kmeans_update(Xg, lab, Cg, C_new=C_new, ctx=ctx)
    assert e.value.code == gb.GBKM_ENOMEM and "injected" in str(e.value)
    ctx.sync()
    assert bool((C_new == -1.0).all())       # nothing was queued
    out = gb.kmeans_update(Xg, lab, Cg, C_new=C_new, ctx=ctx)
    ctx.sync()
    L = lab.cpu().numpy()
    ref = orc.update(X, L, C.astype(np.float64))
    assert centroid_err(out["C_new"].cpu().numpy(), ref["C_new"], X, L) <= CENTROID_REL
    ctx.close()
