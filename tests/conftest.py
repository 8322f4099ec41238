"""Shared pytest configuration: the `gpu` marker and the repository on sys.path."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running statistical test")


import json

import pytest

GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture
def golden():
    """Loader for the cited fixtures under tests/golden/."""
    def load(name):
        with open(os.path.join(GOLDEN, name)) as f:
            return json.load(f)
    return load
