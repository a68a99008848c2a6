import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def tiny():
    """The 10x10 workload: 200 faces, 400 non-faces, seed 1306."""
    from paper_1306_1467_gb300 import synth
    px, y = synth.make_windows(200, 400, 10, 10, seed=1306)
    return px, y


@pytest.fixture(scope="session")
def tiny_prepared(tiny):
    import oracle as O
    px, y = tiny
    return O.Prepared(px, y)
