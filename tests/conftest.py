"""pytest configuration: the `gpu` marker and shared fixtures.

Tests marked `gpu` need a CUDA device and the compiled library; everything
else runs on the CPU (oracle pins, host logic, the C-ABI symbol check).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session")
def oracle():
    from oracle import gdo
    gdo.lib()
    return gdo


@pytest.fixture(scope="session")
def gd():
    """The CUDA library binding (built in-tree); gpu tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35967_gb300 import binding
    binding.load()
    return binding
