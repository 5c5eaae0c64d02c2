import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def glasso():
    """The C-ABI binding (builds the in-tree library first if it is missing)."""
    lib = os.path.join(ROOT, "paper_2205_10027_gb300", "libglasso.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    from paper_2205_10027_gb300 import binding
    return binding


@pytest.fixture(scope="session")
def fp64(glasso):
    """An FP64 handle on cuda:0."""
    h = glasso.Handle(precision="fp64", device=0)
    yield h
    h.close()
