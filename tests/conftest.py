"""pytest configuration: the `gpu` marker and shared helpers.

Tests marked gpu need a CUDA device and the built library; everything else runs on
the CPU (oracle pins, host logic, ABI symbol checks)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built liblbm.so")


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def lbm_lib():
    """The ctypes binding, building liblbm.so first if needed."""
    from paper_2405_12082_gb300 import build
    build.build()
    from paper_2405_12082_gb300 import lbm
    return lbm
