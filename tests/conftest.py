import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# A directory holding another copy of the `oracle` package, imported in its
# place (tests/test_oracle_mutants.py runs the pins against planted mistakes).
_ORACLE_UNDER_TEST = os.environ.get("SL1M_ORACLE_UNDER_TEST")
if _ORACLE_UNDER_TEST:
    sys.path.insert(0, _ORACLE_UNDER_TEST)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled libsl1m")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The compiled CUDA library; GPU tests fail loudly when it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_1310_2078_gb300 import sl1m
    sl1m.load()          # raises if libsl1m.so is missing or fails to load
    return sl1m
