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


def report_err(label, e):
    """Print a measured error in one greppable line (pytest -s shows it);
    the bounds in the tests are set from these lines, ~2x the measured value."""
    print(f"MEASURED_ERR {label} {e:.3e}")
    return e
