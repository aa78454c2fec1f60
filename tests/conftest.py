import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def have_gpu():
    import torch
    return torch.cuda.is_available()


def pytest_sessionstart(session):
    # build the oracle and, where nvcc exists, the CUDA library (no-ops when
    # they are up to date); a missing CUDA library makes the GPU tests fail
    # loudly on import rather than fall back to anything
    import shutil
    from oracle import build as ob
    ob.build()
    if shutil.which("nvcc"):
        from paper_2512_11112_b300 import build as pb
        pb.build()
