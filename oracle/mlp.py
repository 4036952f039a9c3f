"""FP64 reference of the learned candidate proposal's network -- TEST INFRASTRUCTURE ONLY.

The network maps a point x (d_in) to logits over k centers:
    H1 = GELU(x W1^T + b1),  H2 = GELU(H1 W2^T + b2),  z = H2 W3^T + b3,
GELU(t) = t * Phi(t) with Phi the standard normal CDF (erf form).  Training minimises the mean
softmax cross-entropy against exact-method labels with AdamW.  The parameter vector layout is
W1 (h x d_in), b1 (h), W2 (h x h), b2 (h), W3 (k x h), b3 (k) -- the same as the library's.
Plain numpy in float64; the backward pass is written out layer by layer (pinned against
central finite differences of the loss in tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def layout(d_in, h, k):
    sizes = [("W1", (h, d_in)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)), ("W3", (k, h)), ("b3", (k,))]
    out, off = {}, 0
    for name, shp in sizes:
        m = int(np.prod(shp))
        out[name] = (off, shp)
        off += m
    return out, off


def unpack(params, d_in, h, k):
    lay, total = layout(d_in, h, k)
    params = np.asarray(params, np.float64)
    assert params.size == total
    return {n: params[o:o + int(np.prod(s))].reshape(s) for n, (o, s) in lay.items()}


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / np.sqrt(2.0)))


def gelu_grad(t):
    return 0.5 * (1.0 + erf(t / np.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / np.sqrt(2.0 * np.pi)


def forward(params, X, d_in, h, k):
    P = unpack(params, d_in, h, k)
    X = np.asarray(X, np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    H1 = gelu(a1)
    a2 = H1 @ P["W2"].T + P["b2"]
    H2 = gelu(a2)
    z = H2 @ P["W3"].T + P["b3"]
    return {"a1": a1, "H1": H1, "a2": a2, "H2": H2, "z": z}


def loss(params, X, labels, d_in, h, k):
    z = forward(params, X, d_in, h, k)["z"]
    zmax = z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z - zmax).sum(axis=1)) + zmax[:, 0]
    return float(np.mean(lse - z[np.arange(len(labels)), labels]))


def loss_and_grad(params, X, labels, d_in, h, k):
    """Mean softmax cross-entropy and its gradient (same layout as params)."""
    P = unpack(params, d_in, h, k)
    X = np.asarray(X, np.float64)
    B = X.shape[0]
    f = forward(params, X, d_in, h, k)
    z = f["z"]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    L = float(np.mean(np.log(e.sum(axis=1)) + zmax[:, 0] - z[np.arange(B), labels]))
    dz = p.copy()
    dz[np.arange(B), labels] -= 1.0
    dz /= B
    g = {}
    g["W3"] = dz.T @ f["H2"]
    g["b3"] = dz.sum(axis=0)
    dH2 = dz @ P["W3"]
    da2 = dH2 * gelu_grad(f["a2"])
    g["W2"] = da2.T @ f["H1"]
    g["b2"] = da2.sum(axis=0)
    dH1 = da2 @ P["W2"]
    da1 = dH1 * gelu_grad(f["a1"])
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    lay, total = layout(d_in, h, k)
    grad = np.zeros(total)
    for n, (o, s) in lay.items():
        grad[o:o + int(np.prod(s))] = g[n].reshape(-1)
    return L, grad


def adamw_step(params, grad, m, v, step, lr, wd, mask, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (decoupled decay on mask); step is the new step number (1-based)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    p = params - lr * wd * params * mask
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v


def wd_mask(d_in, h, k):
    lay, total = layout(d_in, h, k)
    mask = np.zeros(total)
    for n, (o, s) in lay.items():
        if n.startswith("W"):
            mask[o:o + int(np.prod(s))] = 1.0
    return mask
