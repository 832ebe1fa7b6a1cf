import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def params():
    import oracle
    return oracle.load_params()


@pytest.fixture(scope="session")
def params_rstar():
    """The same derived set fitted with the paper's long cut-off r* = 8.262 A (Sec. 2.6)."""
    import oracle
    return oracle.load_params(os.path.join(ROOT, "paper_1507_07068_gb300", "cr_c_params_rstar.json"))
