import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librtcc.so")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")
    config.addinivalue_line("markers", "last: run after every other selected test (long runs and the newest "
                                       "device paths, so that a stop on failure still leaves the rest reported)")


def pytest_collection_modifyitems(session, config, items):
    """Stable move of the tests marked `last` to the end of the run."""
    items[:] = [i for i in items if i.get_closest_marker("last") is None] + \
               [i for i in items if i.get_closest_marker("last") is not None]
