import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.load()


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, built if needed; fails (never skips) when it cannot load."""
    import torch
    assert torch.cuda.is_available(), "GPU test collected on a machine without a GPU"
    from paper_2509_13230_gb300 import _native, build
    build.build()
    return _native.load()
