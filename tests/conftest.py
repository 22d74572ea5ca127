import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture
def golden_dir():
    return GOLDEN


@pytest.fixture(scope="session")
def cuda():
    """The first CUDA device, with libholo.so built and loaded; fails (no skip) without one."""
    import torch

    assert torch.cuda.is_available(), "a CUDA GPU is required for -m gpu tests"
    from paper_2004_04049_gb300 import build_lib, holo

    build_lib.build()
    holo.load()
    return torch.device("cuda:0")
