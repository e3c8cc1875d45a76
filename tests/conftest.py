import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs of more than a few seconds")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library through its C ABI; a GPU test fails (does not skip)
    when the library or the device is missing."""
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    import paper_1612_07873_gb300 as gb
    return gb
