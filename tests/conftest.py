"""Shared fixtures.  ``gpu`` marks tests that need a CUDA device."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_FACTORS = {}


@pytest.fixture(scope="session")
def oracle_factors():
    """Cached oracle SVD factors keyed by (p, d, eps)."""
    from oracle import m2l

    def get(p, d, eps):
        key = (p, d, eps)
        if key not in _FACTORS:
            _FACTORS[key] = m2l.svd_factors(p, d, eps)
        return _FACTORS[key]

    return get
