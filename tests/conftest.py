import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libv3dg.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def tiny_asset():
    from synth.assets import make_asset
    return make_asset(0, 100_000)


@pytest.fixture(scope="session")
def small_asset():
    from synth.assets import make_asset
    return make_asset(3, 20_000)
