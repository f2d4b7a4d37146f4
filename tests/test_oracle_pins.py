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


def test_count_1e12_golden_is_pinned():
    """The stored 932-bin expectation of the headline count (written by
    tests/golden/make_count_1e12_bins.py from the oracle alone) against the
    published totals pi(10^12) (OEIS A006880) and the sum of the primes below
    10^12 (OEIS A046731), and against the prime number theorem bin by bin."""
    import math

    full = C.golden("count_1e12_bins.json")
    pub = C.golden("pi_powers_of_ten.json")
    bins = full["bins"]
    assert len(bins) == 932 and sum(bins) == full["count"] == pub["pi"]["12"]
    assert full["sum_below_1e12"] == 18435588552550705911377
    assert full["checksum_mod_2_64"] == full["sum_below_1e12"] % 2**64
    w = full["seg_width"]
    for i, b in enumerate(bins[1:-1], start=1):
        # li(x) growth: the count in [a, a + w) lies within 1% of w / ln(a + w / 2) here
        mid = i * w + w / 2
        assert abs(b - w / math.log(mid)) < 0.01 * b, i
    # the first block holds the primes below 2^30: pi(2^30) = 54400028 (OEIS A007053)
    assert bins[0] == 54400028
