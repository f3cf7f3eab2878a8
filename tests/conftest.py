import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs the CUDA path through the C-ABI")


@pytest.fixture(scope="session")
def native_lib():
    """libqkc built in-tree (host compiler + CUDA kernels); loading never needs a GPU."""
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native
    return native.lib()


@pytest.fixture(scope="session")
def cuda_ctx(native_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_2103_17226_gb300 import native
    return native.Context(0)
