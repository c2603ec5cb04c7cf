import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def dense_of(apply, shape_in, n_in=None):
    """Dense matrix of a linear map given as a function on arrays of shape_in."""
    import numpy as np
    n = int(np.prod(shape_in)) if n_in is None else n_in
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape_in))).ravel())
    return np.stack(cols, axis=1)


@pytest.fixture
def dense():
    return dense_of
