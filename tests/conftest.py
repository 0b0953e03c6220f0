import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large workload (minutes of CPU time)")


_BOXES = {}


def cached_config(name):
    """Workload configurations, generated once per test process."""
    from paper_1306_1737_gb300 import workloads as w
    if name not in _BOXES:
        _BOXES[name] = getattr(w, name)()
    return _BOXES[name]


@pytest.fixture(scope="session")
def cfg1():
    return cached_config("config1")


@pytest.fixture(scope="session")
def cfg2():
    return cached_config("config2")
