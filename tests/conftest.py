"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device and the compiled CUDA library; the CPU suite
          runs with ``-m "not gpu"``.
  slow -- longer CPU runs (still part of the default CPU suite).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
