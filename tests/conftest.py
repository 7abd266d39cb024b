import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libkrr")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build_oracle()
    return oracle


def f32(v):
    """The value a float scalar takes at the C boundary (sigma, gamma and the
    shift are float there): the oracle is given exactly the operator the
    library receives."""
    import numpy as np
    return float(np.float32(v))
