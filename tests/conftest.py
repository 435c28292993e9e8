import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def cfg0_literal():
    import ftsynth

    return ftsynth.config0("literal")


@pytest.fixture(scope="session")
def cfg0_auto():
    import ftsynth

    return ftsynth.config0("auto")


@pytest.fixture(scope="session")
def cfg1():
    import ftsynth

    return ftsynth.config1()
