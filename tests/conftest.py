import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: long-running oracle check")


@pytest.fixture(scope="session")
def cuda():
    """The CUDA device with libps.so built; GPU tests fail (not skip) when
    either is missing."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    return dev
