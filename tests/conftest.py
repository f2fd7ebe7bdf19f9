import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running GPU test at full benchmark size")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device; fail loudly instead of skipping
    # silently only when the user explicitly selected them.
    pass
