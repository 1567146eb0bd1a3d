import os
import sys
import functools

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@functools.lru_cache(maxsize=None)
def _event(idx, **kw):
    import synth
    return synth.generate_config(idx, **kw)


@pytest.fixture(scope="session")
def event0():
    return _event(0)


@pytest.fixture(scope="session")
def event1():
    return _event(1)


@pytest.fixture(scope="session")
def oracle0(event0):
    import oracle
    return oracle.track_event(event0)
