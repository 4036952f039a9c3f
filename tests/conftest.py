import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    return oracle


@pytest.fixture(scope="session")
def gb():
    """The CUDA binding, built in-tree; skips only when this machine has no GPU at all."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device on this machine")
    from paper_1502_04265_gb300 import _binding, build

    build.build()
    _binding.load()
    return _binding
