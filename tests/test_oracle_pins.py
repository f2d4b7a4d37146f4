"""The CPU oracle, pinned to published values, the paper's worked example,
exact library routines and independent brute force (see oracle_checks.py)."""
import pytest

import oracle
import oracle_checks as C


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("check", C.ALL_FAST_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(o, check):
    check(o)


def test_oracle_pi_1e10(o):
    """pi(10^10) = 455052511 and the sum of primes below 10^10 (published values)."""
    C.check_range_1e10(o)
