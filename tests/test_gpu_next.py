"""GPU parity of the incremental generator (sieve_next): the primes after a
cursor, with the base table grown by the sieve itself when the walk passes
the square of its limit.  Bit-exact against the CPU oracle."""
import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_first_million_primes(torch):
    with binding.Sieve(10**6) as sv:
        got = sv.next_primes(0, 10**6)
    g = C.golden("pi_powers_of_ten.json")
    assert got.size == 10**6
    assert int(got[-1]) == 15485863  # the millionth prime
    want = oracle.primes_upto(15485863).astype(np.uint64)
    np.testing.assert_array_equal(got, want)
    assert int(np.searchsorted(got, 10**6, side="right")) == g["pi"]["6"]


def test_chained_cursor_equals_one_call(torch):
    with binding.Sieve(10**10) as sv:
        parts, after = [], 10**9
        for _ in range(40):
            p = sv.next_primes(after, 12345)
            parts.append(p)
            after = int(p[-1])
        chained = np.concatenate(parts)
        single = sv.next_primes(10**9, 40 * 12345)
    np.testing.assert_array_equal(chained, single)
    np.testing.assert_array_equal(single, oracle.list_range(10**9 + 1, int(single[-1]) + 1))


def test_table_grows_on_demand(torch):
    with binding.Sieve(1000) as sv:
        lim0, n0, _ = sv.base_table()
        got = sv.next_primes(10**12, 20000)
        lim1, n1, _ = sv.base_table()
        assert lim1 > lim0 and n1 > n0 and lim1 * lim1 >= int(got[-1])
        np.testing.assert_array_equal(got, oracle.list_range(10**12 + 1, int(got[-1]) + 1))
        got2 = sv.next_primes(10**15, 5000)
        lim2, _, _ = sv.base_table()
        assert lim2 * lim2 >= int(got2[-1])
        np.testing.assert_array_equal(got2, oracle.list_range(10**15 + 1, int(got2[-1]) + 1))
        # the grown table still answers ranges below it
        r = sv.range_count(0, 10**8 + 1)
        assert r.count == C.golden("pi_powers_of_ten.json")["pi"]["8"]


def test_device_output_and_edges(torch):
    with binding.Sieve(10**8) as sv:
        out = torch.zeros(3000, dtype=torch.int64, device="cuda")
        n = sv.next_primes(123456789, 3000, out)
        assert n == 3000
        host = sv.next_primes(123456789, 3000)
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), host)
        assert sv.next_primes(5, 0).size == 0
        assert sv.next_primes(1, 3).tolist() == [2, 3, 5]
        assert sv.next_primes(2, 1).tolist() == [3]
        # 2^63 - 25 is the largest prime below 2^63: nothing follows it below 2^63
        with pytest.raises(binding.SieveError) as e:
            sv.next_primes(2**63 - 25, 1)
        assert e.value.status == binding.ERR_RANGE
