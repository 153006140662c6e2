import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


@pytest.fixture(scope="session")
def gpu_lib():
    """The built hvox library on a CUDA device; the GPU tests fail (not skip) without it."""
    import torch
    assert torch.cuda.is_available(), "GPU test collected on a machine without CUDA"
    import paper_2306_06007_gb300 as hvox
    hvox.load()
    return hvox
