"""Shared pytest set-up: repository root on sys.path and the ``gpu`` marker.

Tests marked ``gpu`` need a CUDA device and the compiled library; every other
test runs on the CPU alone.
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU and the compiled rtf library")
