import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def built_lib():
    """Build the CUDA library in-tree (idempotent) and return its path."""
    from paper_2501_10709_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def ctx(built_lib):
    import paper_2501_10709_gb300 as fr
    return fr.fr_ctx_create(0)


@pytest.fixture(scope="session")
def dev():
    import torch
    return torch.device("cuda:0")
