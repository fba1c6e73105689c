"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the built libfb.so; everything else runs
on the CPU (oracle pins, host logic, ABI symbol checks).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and libfb.so")
    config.addinivalue_line("markers", "slow: long-running case")


def read_golden(name):
    """Rows of a golden text fixture, comments stripped, split on whitespace."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows
