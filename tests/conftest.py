import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # The full-size test of the benchmark workload is the longest GPU test: it
    # runs after the other parity tests (and before the test_zz files, which
    # are collected last on purpose); the sort is stable otherwise.
    def key(item):
        name = os.path.basename(str(item.fspath))
        return (name.startswith("test_zz"), name == "test_gpu_fullsize.py")

    items.sort(key=key)
