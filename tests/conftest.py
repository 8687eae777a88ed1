import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    # LBM_ORACLE_UNDER_TEST: a directory holding a copy of the oracle package with one planted
    # mistake (tests/test_oracle_mutants.py), which the pins must then reject
    alt = os.environ.get("LBM_ORACLE_UNDER_TEST")
    if alt:
        sys.path.insert(0, alt)
    import oracle

    if alt:
        assert os.path.dirname(os.path.dirname(os.path.abspath(oracle.__file__))) == alt

    oracle.lib()
    return oracle
