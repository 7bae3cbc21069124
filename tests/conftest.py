import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def fft3d_lib():
    """The C-ABI library, built (incrementally) if needed.  Building needs
    nvcc only, no GPU."""
    from paper_2006_08435_gb300 import build as B, _lib
    B.build()
    return _lib.lib()


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_08435_gb300 import build as B
    B.build()
    return torch.device("cuda:0")
