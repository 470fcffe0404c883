import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (B300, sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: long CPU-side check")


@pytest.fixture(scope="session")
def lib():
    """Build (if stale) and load the CUDA library's binding."""
    from paper_1804_07981_b300 import build as _build
    _build.build()
    from paper_1804_07981_b300 import bml
    return bml


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
