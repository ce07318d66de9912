import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def tiny():
    from paper_2605_01748_b300 import instances
    return instances.make_tiny()


@pytest.fixture(scope="session")
def medium():
    from paper_2605_01748_b300 import instances
    return instances.make_medium()
