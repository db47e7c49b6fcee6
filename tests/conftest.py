"""Test configuration: the ``gpu`` marker and shared fixtures.

``-m "not gpu"`` tests run on a CPU-only machine: the oracle against what the paper
fixes, the host logic, and loading of the CUDA library's exported symbols.
``-m gpu`` tests call the CUDA path through its C ABI and compare with the oracle.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def asx():
    """The CUDA library's Python binding, built in-tree if needed (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14933_gb300 import build as pkg_build
    pkg_build.build()
    import paper_2406_14933_gb300 as pkg
    return pkg
