import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def dcmod():
    """The native package, built in-tree first if needed (nvcc required)."""
    from paper_2311_14312_gb300 import build as B
    B.build()
    import paper_2311_14312_gb300 as P
    return P


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return True
