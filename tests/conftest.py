import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)          # helper modules of the tests (subspace.py)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built hbsd library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def small_problem():
    from paper_1308_2445_gb300 import pufe_inputs
    return pufe_inputs.small_case(1)
