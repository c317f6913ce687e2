import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built librbffd")
    config.addinivalue_line("markers", "slow: long-running case")


def cuda_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lib():
    """The built and loaded C-ABI library (GPU tests only)."""
    if not cuda_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2107_03632_gb300 import rbffd

    return rbffd.load()
