"""Shared pytest configuration.

Markers: ``gpu`` -- needs a CUDA device and the compiled CUDA library; all
other tests run on the CPU (the oracle against its pins, host logic, the
C-ABI symbol table, multi-rank host paths over gloo).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session", autouse=True)
def _build_oracle():
    import oracle
    oracle.build()
    yield
