"""GPU parity of the plain global-bitmap sieve (sieve_range_naive), the
comparison point for the segmented path: counts, checksums and lists against
the CPU oracle and the published values, bit-exact (integer results)."""
import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = binding.Sieve(10**16)
    yield s
    s.close()


EDGES = [(0, 0), (0, 1), (0, 2), (0, 3), (2, 3), (3, 4), (0, 9), (0, 10), (9, 10), (8, 26), (24, 26), (25, 26),
         (1, 2), (0, 100), (49, 50), (121, 122), (10**12, 10**12), (10**12 - 11, 10**12 + 39)]


def test_naive_edges_and_random(sv):
    q = workloads.random_small_ranges(120, seed=31, max_lo=10**13, max_width=300_000)
    ranges = EDGES + list(zip(q.lo.tolist(), q.hi.tolist()))
    for lo, hi in ranges:
        want = oracle.count_range(lo, hi)
        got = sv.naive_count(lo, hi)
        assert (got.count, got.checksum) == want, (lo, hi)
        lst = sv.naive_list(lo, hi)
        assert lst.size == want[0], (lo, hi)
        if want[0]:
            np.testing.assert_array_equal(lst, oracle.list_range(lo, hi))


def test_naive_published_and_plain_range(sv):
    g = C.golden("pi_powers_of_ten.json")
    for e in (6, 8, 10):
        got = sv.naive_count(0, 10**e)
        assert got.count == g["pi"][str(e)] and got.checksum == g["sum_below"][str(e)] % 2**64, e
    lst = sv.naive_list(2, 10**8 + 1)
    assert lst.size == g["pi"]["8"]
    np.testing.assert_array_equal(lst, oracle.list_range(2, 10**8 + 1))
    # far up: windows near 1e15 and 1e16 against the oracle
    for lo in (10**15 - 777, 10**16 - 2_000_001):
        hi = lo + 2_000_000
        got = sv.naive_count(lo, hi)
        assert (got.count, got.checksum) == oracle.count_range(lo, hi), lo
        np.testing.assert_array_equal(sv.naive_list(lo, hi), oracle.list_range(lo, hi))


def test_naive_equals_segmented(sv):
    for lo, hi in ((10**11, 10**11 + 10**9), (3 * 10**12 + 1, 3 * 10**12 + 10**8 + 7)):
        a = sv.naive_count(lo, hi)
        b = sv.range_count(lo, hi)
        assert (a.count, a.checksum) == (b.count, b.checksum), lo


def test_naive_errors(sv):
    with pytest.raises(binding.SieveError) as e:
        sv.naive_count(10, 5)
    assert e.value.status == binding.ERR_INVALID
    with pytest.raises(binding.SieveError) as e:
        sv.naive_count(0, 10**17)
    assert e.value.status == binding.ERR_RANGE
    out = np.zeros(3, dtype=np.uint64)
    with pytest.raises(binding.SieveError) as e:
        sv.naive_list(0, 100, out)
    assert e.value.status == binding.ERR_CAPACITY
