import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


def pytest_sessionstart(session):
    # a fresh checkout has no built library (it is not versioned): build it
    # in-tree before the tests load it (nvcc cross-compiles without a GPU)
    from paper_2404_14044_b300 import build
    for checks in (False, True):
        if not os.path.exists(build.LIB_CHECKS if checks else build.LIB):
            build.build(checks=checks)
