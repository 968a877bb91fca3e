import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def fab():
    """One library context on cuda:0 (GPU tests only)."""
    from paper_2406_17782_gb300 import build as b
    b.build()
    from paper_2406_17782_gb300.api import Fabric
    f = Fabric(0)
    yield f
    f.close()
