import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def golden(name):
    """Values of one line of tests/golden/paper_constants.txt."""
    path = os.path.join(ROOT, "tests", "golden", "paper_constants.txt")
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line and line[0] == name:
                return [float(v) for v in line[1:]]
    raise KeyError(name)
