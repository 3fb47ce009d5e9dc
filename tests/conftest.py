"""Shared fixtures. Tests marked ``gpu`` need a CUDA device and the compiled
library; everything else runs on the CPU (oracle pins, host logic, the ABI
symbol check)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth():
    from paper_1003_1148_gb300 import synth as s
    s.build()
    return s
