"""Shared pytest configuration: the ``gpu`` marker, import paths, and the
release of device memory PyTorch caches between GPU test modules."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")


@pytest.fixture(autouse=True, scope="module")
def _release_cached_device_memory(request):
    """After each GPU test module, hand the memory PyTorch's caching allocator
    keeps from its tests (states of up to 64 GiB) back to the device, so that
    the library's own allocations in later modules (a server's HBM budget,
    the module load of a first launch) find it free."""
    yield
    marks = getattr(request.module, "pytestmark", [])
    marks = marks if isinstance(marks, list) else [marks]
    if not any(getattr(m, "name", "") == "gpu" for m in marks):
        return
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
