import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TABLE_CACHE = os.path.join(ROOT, "oracle", "_build", "cache")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_tables():
    from oracle import tables
    return tables.build_tables(TABLE_CACHE)


@pytest.fixture(scope="session")
def sphere_c1(oracle_tables):
    import synthetic as syn
    from oracle.system import OracleSystem
    prob = syn.sphere_problem(h=0.25)
    return prob, OracleSystem.from_problem(prob, tables=oracle_tables)
