import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session", autouse=True)
def _built_libraries():
    """Compile the oracle and the CUDA library in-tree if they are missing (nvcc
    cross-compiles for sm_103a without a GPU)."""
    import oracle
    oracle.build()
    from paper_2303_10672_b300 import build as cuda_build
    cuda_build.build()
    yield
