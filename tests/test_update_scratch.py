"""The scratch size of the allocation-free update, on the CPU (host arithmetic, no device).

include/gbkm.h states the bytes kmeans_update_noalloc needs as a formula; the library's
kmeans_update_scratch_bytes evaluates its own workspace plan.  The two must agree, so that a
caller sizing problems from the header never meets an unexpected GBKM_ETOOBIG.
"""
import math

import pytest

from paper_1502_04265_gb300 import _binding


def _r256(b):
    return (b + 255) // 256 * 256


def header_formula(n, d, k):
    """The header's formula, written out term by term."""
    r = 256 if k <= 2048 else 128
    while k * math.ceil(n / r) > (1 << 23):
        r *= 2
    S = math.ceil(n / r)
    kS = k * S
    I = math.ceil(n / 128) + k
    terms = [4 * kS, 4 * kS, 4 * math.ceil(kS / 4096), 4 * (k + 1), 4 * (k + 1), 4 * n, 8 * I * d,
             8 * (math.ceil(I / 32) + k) * d, 16 * I, 8 * k * (2 + 2 * math.ceil(d / 256)), 4 * k, 4]
    return 256 + sum(_r256(t) for t in terms)


@pytest.fixture(scope="module")
def lib():
    return _binding.load(build_if_missing=True)


@pytest.mark.parametrize("n,d,k", [(1, 1, 1), (7_001, 37, 13), (30_000, 128, 40), (200_000, 1024, 100),
                                   (20_000, 32, 3_000), (1_000_000, 64, 1_000), (5_000_000, 16, 2_049),
                                   (123_457, 300, 2_048), (40_000, 2_048, 65_536)])
def test_header_formula_matches_the_plan(lib, n, d, k):
    assert _binding.kmeans_update_scratch_bytes(n, d, k) == header_formula(n, d, k)


def test_highdim_workload_needs_about_16_mb(lib):
    b = _binding.kmeans_update_scratch_bytes(200_000, 1024, 100)
    assert 16.2e6 < b < 16.5e6
    assert b <= _binding.NOALLOC_SCRATCH_BYTES


def test_bad_sizes_return_minus_one(lib):
    for n, d, k in [(0, 4, 2), (10, 0, 2), (10, 4, 0), (10, 4, 65_537), (1 << 31, 4, 2)]:
        assert _binding.kmeans_update_scratch_bytes(n, d, k) == -1


def test_update_wrappers_check_shapes_before_any_call():
    """A C_old narrower than d (or an output of the wrong shape) is refused in the binding; the
    checks run before any tensor reaches the library, so CPU tensors serve here."""
    import torch

    X = torch.zeros(10, 8)
    lab = torch.zeros(10, dtype=torch.int32)
    for fn in (_binding.kmeans_update, _binding.kmeans_update_noalloc):
        with pytest.raises(ValueError, match="C_old"):
            fn(X, lab, torch.zeros(3, 7))
        with pytest.raises(ValueError, match="C_new"):
            fn(X, lab, torch.zeros(3, 8), C_new=torch.zeros(3, 7))
        with pytest.raises(ValueError, match="counts"):
            fn(X, lab, torch.zeros(3, 8), counts=torch.zeros(2, dtype=torch.float64))
        with pytest.raises(ValueError, match="labels"):
            fn(X, lab[:9], torch.zeros(3, 8))
