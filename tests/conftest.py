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
def lib():
    """The GPU library through its Python binding (built in-tree on first use)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_01190_gb300 as lcp

    lcp.load()
    return lcp
