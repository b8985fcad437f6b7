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


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print every image/depth parity comparison of the session: pixels
    compared, near decisions, pixels resolved to another branch, pixels two
    branches match, excluded pixels and their fraction, gradient upstream
    zeroed."""
    mod = sys.modules.get("parity")
    log = getattr(mod, "PARITY_LOG", None) if mod else None
    if not log:
        return
    terminalreporter.section("parity: excluded and branch-resolved pixels")
    for s in log:
        terminalreporter.write_line(
            f"{s['label']}: {s['pixels']} px, near {s['near']}, other branch {s['alt_branch']}, "
            f"two branches {s['multi']}, excluded {s['excluded']} ({s['excluded_frac']:.2e}), "
            f"grad upstream zeroed {s.get('grad_zeroed', '-')}, img max {s['img_max']:.2e}, "
            f"depth rel max {s['depth_rel_max']:.2e}")
