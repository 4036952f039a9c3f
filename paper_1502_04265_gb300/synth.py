"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module draws random numbers and nothing else: it holds none of the
k-means arithmetic (no distances, sums, argmins or projections of the method).
Both sides of every parity test receive the arrays it returns.

The paper's datasets (Caltech128, BagOfWords, Covertype, BigCross; Section 3)
are not available, so seeded Gaussian mixtures shaped like the paper's
high-dimensional workloads stand in for them:

  1. mixture weights  pi ~ Dirichlet(1, ..., 1)
  2. means            mu_j ~ U[-10, 10]^d
  3. spreads          sigma_j = exp(U[ln 0.5, ln 2])
  4. components       z_i ~ Categorical(pi)
  5. points           x_i = mu_{z_i} + sigma_{z_i} * N(0, I_d)

drawn in that order from numpy's PCG64 ``default_rng(seed)``.  The
low-rank-subspace workload embeds such a mixture in a random orthonormal
rank-r basis Q and adds isotropic noise (the data model behind the
best-fit-subspace projection of Section 2.2).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gaussian_mixture",
    "seed_uniforms",
    "integer_weights",
    "orthonormal_basis",
    "subspace_mixture_chunk",
    "batch_problem_list",
    "mlp_init",
    "bico_members",
    "bico_batch",
]


def gaussian_mixture(n: int, d: int, n_comp: int, seed: int, *, chunk_rows: int = 1 << 16,
                     return_params: bool = False):
    """Draw n points in R^d from the seeded n_comp-component mixture (FP32, row-major).

    Normal draws are made in float32 in chunks of ``chunk_rows`` rows so that
    large workloads (200,000 x 1,024) need no float64 staging copy.
    """
    rng = np.random.default_rng(seed)
    pi = rng.dirichlet(np.ones(n_comp))
    mu = rng.uniform(-10.0, 10.0, size=(n_comp, d)).astype(np.float32)
    sigma = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=n_comp)).astype(np.float32)
    z = rng.choice(n_comp, size=n, p=pi).astype(np.int32)
    X = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        zz = z[r0:r1]
        noise = rng.standard_normal((r1 - r0, d), dtype=np.float32)
        X[r0:r1] = mu[zz] + sigma[zz, None] * noise
    if return_params:
        return X, z, {"pi": pi, "mu": mu, "sigma": sigma}
    return X, z


def structured_with_noise(ell: int, y: int, d: int, x: int, seed: int, *, big: float = 10.0,
                          small: float = 0.5):
    """The StructuredWithNoise instances of Section 3: ell hidden point sets of y points in R^d.

    Cluster i draws x of the d dimensions uniformly without replacement; each of its points takes
    those coordinates uniformly from [-big, big] and every other coordinate uniformly from
    [-small, small] (the paper fixes big = 10, small = 1/2).  Returns X (ell * y x d, FP32, the
    clusters one after another) and the cluster of every row.
    """
    rng = np.random.default_rng([seed, 0x5A7])
    X = np.empty((ell * y, d), dtype=np.float32)
    z = np.repeat(np.arange(ell, dtype=np.int32), y)
    for i in range(ell):
        dims = rng.choice(d, size=x, replace=False)
        blk = X[i * y:(i + 1) * y]
        blk[:] = rng.random((y, d), dtype=np.float32)
        blk *= np.float32(2 * small)
        blk -= np.float32(small)
        blk[:, dims] = (rng.random((y, x), dtype=np.float32) * np.float32(2) - np.float32(1)) * np.float32(big)
    return X, z


def seed_uniforms(k: int, seed: int) -> np.ndarray:
    """The k uniforms in [0, 1) that drive one k-means++ run (FP64).

    u[0] picks the first center, u[j] the (j+1)-th; the method's random draws
    are inputs so that the oracle and the GPU consume the same stream.
    """
    rng = np.random.default_rng([seed, 0x5EED])
    return rng.random(k)


def integer_weights(n: int, seed: int, max_w: int = 5) -> np.ndarray:
    """Positive integral point weights (FP32), the kind a coreset carries (Section 2.3.2)."""
    rng = np.random.default_rng([seed, 0x3E16])
    return rng.integers(1, max_w + 1, size=n).astype(np.float32)


def orthonormal_basis(d: int, r: int, seed: int) -> np.ndarray:
    """A random d x r matrix with orthonormal columns (QR of a Gaussian), FP64."""
    rng = np.random.default_rng([seed, 0x0B5])
    G = rng.standard_normal((d, r))
    Q, R = np.linalg.qr(G)
    # fix the sign convention so that the basis is a deterministic function of the seed
    Q = Q * np.sign(np.diag(R))[None, :]
    return Q


def gaussian_sketch(d: int, s: int, seed: int) -> np.ndarray:
    """A d x s matrix of independent N(0, 1) draws, FP32: the random matrix a randomised SVD
    multiplies a piece by (drawn here and passed in, so every implementation uses the same one)."""
    rng = np.random.default_rng([seed, 0x5C7])
    return rng.standard_normal((d, s), dtype=np.float32)


def planted_spectrum(n: int, d: int, sigmas, seed: int) -> np.ndarray:
    """U diag(sigmas) W^T with random orthonormal U (n x r) and W (d x r), FP64: a matrix whose
    singular values are exactly `sigmas` (r = len(sigmas)) and whose right singular vectors are W."""
    sig = np.asarray(sigmas, dtype=np.float64)
    r = sig.shape[0]
    U = orthonormal_basis(n, r, seed * 2 + 1)
    W = orthonormal_basis(d, r, seed * 2 + 2)
    return (U * sig[None, :]) @ W.T


def subspace_mixture_chunk(Q: np.ndarray, row0: int, rows: int, n_comp: int, seed: int,
                           noise: float = 0.1):
    """Rows [row0, row0+rows) of the rank-r-subspace workload, FP32.

    Latent coordinates Z come from an n_comp-component mixture in R^r (the
    five-step recipe above, mixture parameters drawn from ``seed``); each chunk
    draws its own components and noise from ``[seed, row0]`` so that chunks can
    be produced independently.  X = Z Q^T + N(0, noise^2 I_d).
    """
    d, r = Q.shape
    prng = np.random.default_rng(seed)
    pi = prng.dirichlet(np.ones(n_comp))
    mu = prng.uniform(-10.0, 10.0, size=(n_comp, r))
    sigma = np.exp(prng.uniform(math.log(0.5), math.log(2.0), size=n_comp))
    rng = np.random.default_rng([seed, row0])
    z = rng.choice(n_comp, size=rows, p=pi).astype(np.int32)
    Z = mu[z] + sigma[z, None] * rng.standard_normal((rows, r))
    X = Z @ Q.T + noise * rng.standard_normal((rows, d))
    return X.astype(np.float32), z


def batch_problem_list(count: int, seed: int = 0, *, n_range=(1_000, 100_000),
                       d_choices=(32, 128, 512), k_range=(4, 256)):
    """Draw the shapes of ``count`` independent problems (batched workload).

    n and k are log-uniform in their ranges (rounded), d is uniform over
    ``d_choices``; each problem's data seed is its index.
    """
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = int(rng.choice(np.asarray(d_choices)))
        k = int(round(math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1])))))
        k = max(1, min(k, n))
        out.append({"n": n, "d": d, "k": k, "seed": p})
    return out


def mlp_init(d_in: int, hidden: int, k: int, seed: int) -> np.ndarray:
    """Initial parameters of the candidate-proposal network (FP32 vector, layout W1, b1, W2, b2,
    W3, b3 with rows = output units): weights uniform in +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng([seed, 0x31F])
    parts = []
    for fan_out, fan_in in ((hidden, d_in), (hidden, hidden), (k, hidden)):
        bound = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def bico_members(refs: np.ndarray, seed: int, max_members: int = 8):
    """Member points of a snapshot of BICO-style features (Section 2.1), one feature per reference
    row: feature j holds its reference point and N_j - 1 more points around it, N_j uniform in
    {1, ..., max_members}, at a spread sigma_j log-uniform in [0.05, 1] (FP32).  Returns (P, f) with
    f[i] the feature of member P[i]; the features' sums are left to the caller."""
    refs = np.asarray(refs, dtype=np.float32)
    m, d = refs.shape
    rng = np.random.default_rng([seed, 0xB1C0])
    cnt = rng.integers(1, max_members + 1, size=m)
    sig = np.exp(rng.uniform(math.log(0.05), 0.0, size=m)).astype(np.float32)
    f = np.repeat(np.arange(m, dtype=np.int32), cnt)
    noise = rng.standard_normal((f.shape[0], d), dtype=np.float32)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    noise[first] = 0.0
    P = refs[f] + sig[f, None] * noise
    return P.astype(np.float32), f


def bico_batch(refs: np.ndarray, n: int, seed: int):
    """A batch of n points arriving at a BICO-style summary: each lies near a reference row chosen
    uniformly, at a spread of 0.01, 0.3 or 2 (equally likely), so that some points fit their feature
    whole, some in part and some not at all.  FP32."""
    refs = np.asarray(refs, dtype=np.float32)
    m, d = refs.shape
    rng = np.random.default_rng([seed, 0xB1C1])
    j = rng.integers(0, m, size=n)
    sp = np.array([0.01, 0.3, 2.0], np.float32)[rng.integers(0, 3, size=n)]
    X = refs[j] + sp[:, None] * rng.standard_normal((n, d), dtype=np.float32)
    return X.astype(np.float32)
