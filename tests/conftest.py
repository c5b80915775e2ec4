import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libscgr.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def scgr_lib():
    """The CUDA library, built in-tree if needed; the GPU tests call it through the C ABI."""
    from paper_1902_01061_gb300 import build, scgr
    build.build()
    return scgr.load()
