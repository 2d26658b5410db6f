import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


_WL = {}


def workload(name, **kw):
    """Session-cached synthetic workload (bands are generated once per process)."""
    from synth import make_workload
    key = (name, tuple(sorted(kw.items())))
    if key not in _WL:
        _WL[key] = make_workload(name, **kw)
    return _WL[key]


@pytest.fixture(scope="session")
def micro():
    return workload("micro")


@pytest.fixture(scope="session")
def small():
    return workload("small")
