import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def agf2_lib():
    """The built C-ABI library via its ctypes binding (builds it if needed)."""
    from paper_2106_03508_gb300 import build as b
    b.build()
    from paper_2106_03508_gb300 import agf2
    return agf2


@pytest.fixture(scope="session")
def cuda_handle(agf2_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    h = agf2_lib.Handle(0)
    yield h
    h.close()
