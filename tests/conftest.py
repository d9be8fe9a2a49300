import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhpt.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def hpt():
    """The CUDA library's binding; the library is built if needed.  Fails (does
    not skip) when it cannot be built or loaded."""
    from paper_2111_14317_gb300 import build
    build.build()
    from paper_2111_14317_gb300 import hpt as mod
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return mod
