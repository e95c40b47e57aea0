import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbrt.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def lib():
    """Build liblbrt.so in-tree if needed and load it (CPU-safe: no CUDA call)."""
    from paper_2007_05718_gb300 import build, lbrt
    build.build()
    return lbrt.load()


@pytest.fixture(scope="session")
def cuda(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return torch.device("cuda:0")
