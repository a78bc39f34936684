import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def f32(x):
    """A parameter as the library sees it: rounded to float32, then widened."""
    return float(np.float32(x))


@pytest.fixture(scope="session")
def root():
    return ROOT
