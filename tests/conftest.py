import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libcbs.so")
    config.addinivalue_line("markers", "slow: takes tens of seconds")


@pytest.fixture(scope="session")
def built_lib():
    """Compile libcbs.so in-tree (nvcc cross-compiles without a GPU) and return its path."""
    from paper_2506_15411_gb300 import build
    return build.build()
