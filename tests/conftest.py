import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


import pytest


@pytest.fixture(scope="session")
def built_lib():
    """Build libsar.so (nvcc cross-compiles without a GPU) and return its path."""
    import __graft_entry__
    return __graft_entry__._build_module().build()
