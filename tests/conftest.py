import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: minutes of CPU; runs only with TT_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("TT_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle pin: set TT_SLOW=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)
