import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_tables_small():
    """64x64 tables with the paper's axis ranges (§4 benchmark ranges)."""
    import oracle
    return oracle.tables(qs_n_chi=64, qs_n_xi=64, bw_n_chi=64, bw_n_xi=64)


@pytest.fixture(scope="session")
def oracle_tables_256():
    """256x256 tables: chi in [1e-3, 1e3] (QS), [2e-2, 1e3] (BW), xi_min 1e-12 (§4)."""
    import oracle
    return oracle.tables()
