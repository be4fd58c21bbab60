import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: large CPU-side cases")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def built_lib():
    """Build libdd.so (by path, before the package is imported) and return the package."""
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1111_6399_gb300
    return paper_1111_6399_gb300
