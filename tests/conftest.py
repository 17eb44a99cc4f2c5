"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device (GB300, sm_103a); run with ``-m gpu``.
  slow -- CPU tests that take more than ~20 s (still part of ``-m "not gpu"``).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
