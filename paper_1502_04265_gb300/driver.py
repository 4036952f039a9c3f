"""k-means++ then Lloyd's algorithm (Section 1) through the C ABI.

The loop only sequences ABI calls on one stream; every step runs in the
library's kernels.  Stopping rule (the paper allows convergence, a fixed
count, or a small decrease): a fixed number of iterations, as the workloads
specify; the iteration at which the labels stopped changing is reported.
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
          return_trace=False):
    """Seed with k-means++ (unless C0 is given), then run `iters` Lloyd iterations.

    compute: "f32", "bf16", "fp8", or "auto" (exact_form of the dimension).

    Returns a dict with C (k x d), labels, the device cost trace
    [cost(C_t, L_t), cost(C_{t+1}, L_t)] per iteration and the seeding indices.
    """
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
    for t in range(iters):
        B.kmeans_assign(X, C, Xop=Xop, Xop_scales=scales, xnorm=xnorm, compute=compute,
                        engine=engine, labels=labels, n_rechecked=nre[t:t + 1], ctx=ctx)
        B.kmeans_update(X, labels, C, w=w, C_new=C_next, cost_old=trace[t, 0:1],
                        cost_new=trace[t, 1:2], ctx=ctx)
        C, C_next = C_next, C
    out = {"C": C, "labels": labels, "seed_idx": idx}
    if return_trace:
        out["trace"] = trace[:iters]
        out["n_rechecked"] = nre[:iters]
    return out
