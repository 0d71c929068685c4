import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libipt.so")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ipt():
    """The native binding; GPU tests fail loudly when the library is missing."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2012_14702_gb300 import ipt as _ipt
    return _ipt
