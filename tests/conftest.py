"""Shared test configuration.

Markers: ``gpu`` -- needs a CUDA device (run on the GB300 machine); everything
else runs on the CPU.  The oracle and the input generators are compiled on
first use (gcc only).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def vg():
    import volgen
    return volgen
