import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, loaded through the package binding. Fails (does not
    skip) when the extension or the GPU is missing on a GPU run."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test collected but CUDA is not available")
    from paper_2411_19588_b300 import _abi
    return _abi.lib()
