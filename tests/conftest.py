import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle work of more than a few seconds")


@functools.lru_cache(maxsize=None)
def oracle_plan(N, L, tol):
    """Oracle plans are deterministic; tests share them within one session."""
    from oracle import gtensor
    return gtensor.make_plan(N, L, tol)


@functools.lru_cache(maxsize=4)
def oracle_symbol(N, L, tol):
    from oracle import gtensor
    return gtensor.symbol(oracle_plan(N, L, tol))


@pytest.fixture(scope="session")
def plan_cache():
    return oracle_plan


@pytest.fixture(scope="session")
def symbol_cache():
    return oracle_symbol
