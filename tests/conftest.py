"""Shared fixtures.  GPU tests carry the `gpu` marker; everything else runs
on a CPU-only machine."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS_DIR = os.path.dirname(os.path.abspath(__file__))
if TESTS_DIR not in sys.path:
    sys.path.insert(0, TESTS_DIR)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built liblbfd.so")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lbfd_lib():
    """The CUDA library, built in-tree if needed; on a GPU machine its
    absence is an error, never a skip."""
    from paper_2304_05657_gb300 import build, lbfd

    build.build()
    return lbfd
