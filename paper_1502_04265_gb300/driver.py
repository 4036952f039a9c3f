"""k-means++ then Lloyd's algorithm (Section 1) through the C ABI.

The loop only sequences ABI calls on one stream; every step runs in the
library's kernels.  Stopping rule (the paper allows convergence, a fixed
count, or a small decrease): a fixed number of iterations by default, as the
workloads specify, with no host synchronisation; or, with `tol`, the first
iteration whose relative cost decrease is at most tol (0: convergence).  The
iteration at which the cost stopped changing is reported with the trace.
"""
from __future__ import annotations

import torch

from . import _binding as B


# below this dimension BF16's certified band holds most points of typical data, and their FP32
# recheck costs more than the halved read of X saves
BF16_MIN_D = 256


def exact_form(d):
    """The faster of the two exact assignment forms for points of dimension d: "bf16" (with the
    certified recheck) from BF16_MIN_D up when the tensor-core engine takes the shape (d a
    multiple of 8), "f32" otherwise."""
    return "bf16" if d >= BF16_MIN_D and d % 8 == 0 else "f32"


def lloyd(X, k, iters, u, w=None, compute="f32", engine="auto", C0=None, ctx=None,
          return_trace=False, tol=None):
    """Seed with k-means++ (unless C0 is given), then run at most `iters` Lloyd iterations.

    compute: "f32", "bf16", "fp8", or "auto" (exact_form of the dimension).
    tol: None runs exactly `iters` iterations without any host synchronisation.  A number >= 0 ends
    the run after the first iteration whose relative decrease
    (cost(C_t, L_t) - cost(C_{t+1}, L_t)) / cost(C_t, L_t) is at most tol, reading that iteration's
    two costs back (one synchronisation per iteration); tol = 0 stops at convergence, since
    unchanged labels give the same centers and equal costs.

    Returns a dict with C (k x d), labels, the seeding indices and the number of iterations run;
    with return_trace also the device cost trace [cost(C_t, L_t), cost(C_{t+1}, L_t)] per
    iteration, the recheck counts, and converged_at: the first iteration whose update left the cost
    unchanged (None if none did; the trace is read back once, at the end, to find it).
    """
    if tol is not None and not tol >= 0:
        raise ValueError("tol must be None or a number >= 0")
    n, d = X.shape
    dev = X.device
    if compute == "auto":
        compute = exact_form(d)
    idx = None
    xnorm = B.kmeans_row_norms(X, ctx=ctx)
    Xop, scales = (None, None)
    if compute in ("bf16", "fp8"):
        Xop, scales = B.kmeans_quantize(X, compute, ctx=ctx)
    if C0 is None:
        idx, C = B.kmeans_seed_pp(X, k, u, w=w, ctx=ctx)
    else:
        C = C0.clone()
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    C_next = torch.empty_like(C)
    trace = torch.empty((max(iters, 1), 2), dtype=torch.float64, device=dev)
    nre = torch.zeros(max(iters, 1), dtype=torch.int64, device=dev)
    done = iters
    for t in range(iters):
        B.kmeans_assign(X, C, Xop=Xop, Xop_scales=scales, xnorm=xnorm, compute=compute,
                        engine=engine, labels=labels, n_rechecked=nre[t:t + 1], ctx=ctx)
        B.kmeans_update(X, labels, C, w=w, C_new=C_next, cost_old=trace[t, 0:1],
                        cost_new=trace[t, 1:2], ctx=ctx)
        C, C_next = C_next, C
        if tol is not None:
            c_old, c_new = trace[t].tolist()
            if c_old - c_new <= tol * c_old:
                done = t + 1
                break
    out = {"C": C, "labels": labels, "seed_idx": idx, "iterations": done}
    if return_trace:
        out["trace"] = trace[:done]
        out["n_rechecked"] = nre[:done]
        flat = (trace[:done, 0] == trace[:done, 1]).nonzero()
        out["converged_at"] = int(flat[0, 0]) if flat.numel() else None
    return out
