"""The StructuredWithNoise generator (Section 3) against its definition (no GPU)."""
import numpy as np

from paper_1502_04265_gb300 import synth


def test_structured_with_noise_definition():
    ell, y, d, x = 6, 40, 30, 4
    X, z = synth.structured_with_noise(ell, y, d, x, seed=3)
    assert X.shape == (ell * y, d) and X.dtype == np.float32
    assert np.array_equal(z, np.repeat(np.arange(ell), y))
    for i in range(ell):
        rows = X[z == i]
        big = np.abs(rows) > 0.5
        # exactly x dimensions carry the cluster's signal: the same x columns in every row
        sig = np.flatnonzero(big.any(axis=0))
        assert len(sig) <= x
        noise = np.setdiff1d(np.arange(d), sig)
        assert np.all(np.abs(rows[:, noise]) <= 0.5)
        assert np.all(np.abs(rows) <= 10.0)
        # with 40 uniform draws in [-10, 10] every signal column leaves [-1/2, 1/2] somewhere
        assert len(sig) == x
    # deterministic in the seed, different across seeds
    X2, _ = synth.structured_with_noise(ell, y, d, x, seed=3)
    X3, _ = synth.structured_with_noise(ell, y, d, x, seed=4)
    assert np.array_equal(X, X2) and not np.array_equal(X, X3)
