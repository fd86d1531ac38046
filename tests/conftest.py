import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer host-side case")


@pytest.fixture(scope="session")
def tiny():
    import synth
    return synth.make_system("tiny_L6_12")


@pytest.fixture(scope="session")
def cfg24():
    import synth
    return synth.make_system("chi0_L10_24")
