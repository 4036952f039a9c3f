"""Pins of the FP64 MLP oracle: backward pass vs central finite differences of the loss, GELU vs
the normal CDF, AdamW first step in closed form."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_x_phi():
    t = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(t), t * norm.cdf(t), rtol=1e-12, atol=1e-14)
    # derivative by central differences
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(t), (mlp.gelu(t + h) - mlp.gelu(t - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    d_in, h, k, B = 4, 5, 3, 7
    _, total = mlp.layout(d_in, h, k)
    params = rng.normal(size=total) * 0.7
    X = rng.normal(size=(B, d_in))
    y = rng.integers(0, k, size=B)
    L, g = mlp.loss_and_grad(params, X, y, d_in, h, k)
    assert L == pytest.approx(mlp.loss(params, X, y, d_in, h, k), rel=1e-14)
    eps = 1e-6
    fd = np.empty(total)
    for i in range(total):
        e = np.zeros(total)
        e[i] = eps
        fd[i] = (mlp.loss(params + e, X, y, d_in, h, k) - mlp.loss(params - e, X, y, d_in, h, k)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_adamw_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, -1.0, 2.0])
    mask = np.array([1.0, 0.0, 1.0, 0.0])
    lr, wd = 0.01, 0.1
    q, m, v = mlp.adamw_step(p, g, np.zeros(4), np.zeros(4), 1, lr, wd, mask)
    # step 1: mhat = g, vhat = g^2 -> update lr * g / (|g| + eps); decay lr * wd * p on masked entries
    expect = p - lr * wd * p * mask - lr * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(q, expect, rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
