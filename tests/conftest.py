import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


def golden_values(name: str, state: int = 0):
    """Stored oracle results of a full-size workload (tests/golden/oracle_*.txt,
    written by tests/golden/make_oracle_golden.py from the oracle alone)."""
    import numpy as np
    a = np.loadtxt(os.path.join(ROOT, "tests", "golden", f"oracle_{name}_s{state}.txt"), comments="#")
    return a[:, 0] + 1j * a[:, 1]


@pytest.fixture(scope="session")
def golden():
    return golden_values


@pytest.fixture(scope="session")
def orc():
    import oracle
    alt = os.environ.get("TBPM_ORACLE_LIB")   # a planted-mistake build (mutation tests)
    return oracle.Oracle(alt) if alt else oracle.default()
