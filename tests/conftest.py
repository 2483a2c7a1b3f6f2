import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger cases")


@pytest.fixture(scope="session")
def wdlib():
    """Build (if stale) and load the solver library."""
    from paper_2007_01541_gb300 import build as wdbuild
    import paper_2007_01541_gb300 as wd

    wdbuild.build()
    return wd


@pytest.fixture(scope="session")
def cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch
