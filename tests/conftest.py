import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblp")
    config.addinivalue_line("markers", "slow: full-size workload (minutes of CPU oracle time)")


def pytest_collection_modifyitems(config, items):
    # Keep files in name order so test_zz_* files run last.
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)), 0))
