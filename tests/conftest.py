import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built sm_103a library")
    config.addinivalue_line("markers", "slow: longer CPU pin (still part of the default CPU run)")


@pytest.fixture(scope="session")
def cuda_dev():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="session")
def S(cuda_dev):
    # the CUDA library must load on a GPU run: a missing build is an error, not a skip
    import paper_2402_08134_gb300 as lib

    return lib
