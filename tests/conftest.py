import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); calls the CUDA path through the C ABI")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    # the library under test is compiled in-tree; build it (incrementally) if a fresh checkout lacks it
    from paper_2007_00745_gb300 import build as mbuild
    mbuild.build()
    # guard: no test launch may run longer than this (its CTAs stop and set status bit 4)
    import paper_2007_00745_gb300 as mb
    mb.DEFAULT_MAX_SECONDS = 300


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
