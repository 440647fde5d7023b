"""Shared pytest setup: the ``gpu`` marker, import paths and build steps."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (parity tests of the CUDA path)")
    config.addinivalue_line(
        "markers", "slow: full-size parity cases (minutes)")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """Compile the generator and oracle shared objects once per session."""
    import oracle
    import synth
    synth.build()
    oracle.build()
    yield
