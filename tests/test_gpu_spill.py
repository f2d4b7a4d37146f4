"""Long runs that survive interruption (the paper's future-work item 1,
Section 6): a checkpointed count of [2, 1e11] stopped twice and resumed in
fresh contexts must give bit-identical totals and per-block counts to an
uninterrupted run (and the published pi(1e11)); a list spilled to a file in
store segments, interrupted and resumed after garbage was appended to the
file, must equal the CPU oracle's list."""
import os

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


def test_checkpointed_count_resumes_bit_identical(torch, tmp_path):
    lo, hi, w, chunk = 2, 10**11 + 1, 1 << 30, 10**10
    state = str(tmp_path / "count.state")
    with binding.Sieve(hi) as sv:
        done, part, bins, nxt = sv.count_checkpointed(lo, hi, w, chunk, state, max_chunks=4)
        assert not done and nxt == lo + 4 * chunk
    with binding.Sieve(hi) as sv:  # a new process would start like this
        done, part2, bins2, nxt = sv.count_checkpointed(lo, hi, w, chunk, state, max_chunks=3)
        assert not done and nxt == lo + 7 * chunk and part2.count > part.count
    with binding.Sieve(hi) as sv:
        done, tot, bins, nxt = sv.count_checkpointed(lo, hi, w, chunk, state)
        assert done and nxt == hi
        ref, rbins = sv.segment_counts(lo, hi, w)
        again = sv.count_checkpointed(lo, hi, w, chunk, state)  # finished: answered from the state
        # another job's parameters with the same state file are refused
        with pytest.raises(binding.SieveError):
            sv.count_checkpointed(lo, hi, w, chunk // 2, state)
        damaged = str(tmp_path / "damaged.state")
        with open(state, "rb") as f:
            data = bytearray(f.read())
        data[20] ^= 1
        with open(damaged, "wb") as f:
            f.write(data)
        with pytest.raises(binding.SieveError):
            sv.count_checkpointed(lo, hi, w, chunk, damaged)
    g = C.golden("pi_powers_of_ten.json")
    assert tot.count == ref.count == g["pi"]["11"]
    assert tot.checksum == ref.checksum == g["sum_below"]["11"] % 2**64
    np.testing.assert_array_equal(bins, rbins)
    assert again[0] and (again[1].count, again[1].checksum) == (tot.count, tot.checksum)
    np.testing.assert_array_equal(again[2], bins)


def test_spill_to_file_resumes(torch, tmp_path):
    lo, hi = 10**12 - 12345, 10**12 + 10**8
    path = str(tmp_path / "primes.u64")
    with binding.Sieve(hi) as sv:
        done, n1 = sv.primes_to_file(lo, hi, path, segment_primes=500_000, max_segments=5)
        assert not done and n1 > 0 and os.path.getsize(path) == 8 * n1
        with open(path, "ab") as f:  # what an interrupted segment could leave behind
            f.write(b"\x07" * 1000)
        done, n = sv.primes_to_file(lo, hi, path, segment_primes=500_000, resume=True)
        assert done
        # a fresh run (resume off) gives the same file
        path2 = str(tmp_path / "primes2.u64")
        done2, n2 = sv.primes_to_file(lo, hi, path2, segment_primes=1 << 20)
        assert done2 and n2 == n
    got = np.fromfile(path, dtype="<u8")
    want = oracle.list_range(lo, hi)
    assert got.size == n == want.size
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(np.fromfile(path2, dtype="<u8"), want)
