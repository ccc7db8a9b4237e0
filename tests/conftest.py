import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on a GB300 box)")
    config.addinivalue_line("markers", "slow: long CPU-side check")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def fb():
    """The CUDA library binding (GPU tests only)."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    from paper_2004_09883_gb300 import fbfft
    return fbfft
