import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle or GPU case")


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a gpu-marked test ran without a CUDA device")
    return torch.device("cuda:0")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Every measured error of the GPU parity tests, one line each, so that a
    plain `pytest -q` run records them."""
    try:
        import _helpers
    except ImportError:
        return
    if _helpers.PARITY_LOG:
        terminalreporter.section("measured errors against the oracle")
        for line in _helpers.PARITY_LOG:
            terminalreporter.write_line(line)
