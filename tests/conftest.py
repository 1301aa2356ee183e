"""Shared test configuration.

Markers: ``gpu`` tests need a CUDA device and the compiled library; every
other test runs on the CPU (the oracle against its pins, host logic, and the
C-ABI symbol table).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled gwn library")


@pytest.fixture(scope="session")
def cuda_available():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True
