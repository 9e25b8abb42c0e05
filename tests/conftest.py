import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built library")


@pytest.fixture(scope="session")
def nlmg_lib():
    """Builds (if stale) and loads libnlmg.so."""
    from paper_2005_01275_gb300 import build, nlmg
    build.build()
    return nlmg
