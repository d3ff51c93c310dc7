import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def rel_err(a, b):
    """||a - b|| / ||b|| over the concatenation of several arrays."""
    import numpy as np
    a = np.concatenate([np.ravel(np.asarray(x, dtype=np.float64)) for x in a])
    b = np.concatenate([np.ravel(np.asarray(x, dtype=np.float64)) for x in b])
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture
def relerr():
    return rel_err
