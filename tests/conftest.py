import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libcmrs.so")
    config.addinivalue_line("markers", "slow: full-size workload")


def load_golden(name):
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = np.array([float(t) for t in v.split()])
    return out


@pytest.fixture(scope="session")
def golden5():
    return load_golden("paper_5x5.txt")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
