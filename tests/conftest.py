import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device and the compiled correlator library")


@pytest.fixture(scope="session")
def lib():
    """The loaded C-ABI library (built on demand)."""
    from paper_1102_0148_gb300 import corr
    return corr
