"""The entry point that allocates nothing (sieve_range_list_noalloc), called
through the C ABI.  It exists for callers that cannot allocate device memory
when they need primes (their device memory belongs to another allocator, or
cudaMalloc / cudaFree's cost and implicit synchronisation are not allowed);
its scratch is one fixed array in the library's device image, shared by every
call.  Checked against the CPU oracle and against the regular list call
(sieve_range in list mode): exact equality of the lists, counts and
checksums, on calls in a row that share the fixed array, and on edge ranges.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2310_17746_gb300 import binding

pytestmark = pytest.mark.gpu

# ranges of up to this many numbers always fit the fixed scratch with the
# default tile length (2^19 candidates per class)
MAX_WIDTH_DEFAULT_TILE = 399_507_452


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check(sv, torch, lo, hi, base):
    want = oracle.list_range(lo, hi, base=base)
    wc, ws = oracle.count_range(lo, hi, base=base)
    out = torch.full((want.size + 64,), -1, dtype=torch.int64, device="cuda")
    n, cs = sv.range_list_noalloc(lo, hi, out)
    torch.cuda.synchronize()
    assert n == want.size == wc, (lo, hi)
    assert (cs.count, cs.checksum) == (wc, ws), (lo, hi)
    got = out[:n].cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, want), (lo, hi)
    assert bool((out[n:] == -1).all()), (lo, hi)  # nothing written past the list
    return got


def test_no_alloc_list_matches_oracle_and_regular_list():
    torch = _need_gpu()
    base = oracle.base_table(10**6 + 100)
    with binding.Sieve(10**12 + 10**8) as sv:
        # two calls in a row: a wide range near 1e12, then a narrower one from 0 whose
        # tiles reuse (and must overwrite) what the first call left in the scratch
        for lo, hi in ((10**12 - 50_000_000, 10**12 + 40_000_000), (0, 3_000_000)):
            got = _check(sv, torch, lo, hi, base)
            assert np.array_equal(got, sv.range_list(lo, hi))


def test_no_alloc_edge_ranges():
    torch = _need_gpu()
    base = oracle.base_table(10**6 + 100)
    p = 999983  # the largest prime below 1e6: its square lies just under 1e12
    edges = [(0, 0), (10**9 + 7, 10**9 + 7), (0, 2), (2, 3), (3, 5), (0, 6), (1, 7), (24, 29),
             (10**12 - 5, 10**12 + 1), (10**11 + 1, 10**11 + 6),
             (p * p - 5, p * p + 5), (p * p - 6 * 524288, p * p + 3),
             (49 - 5, 49 + 5), (121 - 5, 121 + 5), (113 * 113 - 5, 113 * 113 + 5)]
    with binding.Sieve(10**12 + 10**8) as sv:
        for lo, hi in edges:
            _check(sv, torch, lo, hi, base)


def test_no_alloc_limits():
    torch = _need_gpu()
    with binding.Sieve(10**12) as sv:
        out = torch.zeros(16, dtype=torch.int64, device="cuda")
        with pytest.raises(binding.SieveError) as e:
            sv.range_list_noalloc(0, 10**10, out)
        assert e.value.status == binding.ERR_INVALID
        msg = binding.last_error()
        assert "scratch" in msg and str(MAX_WIDTH_DEFAULT_TILE) in msg, msg
        with pytest.raises(binding.SieveError) as e:
            sv.range_list_noalloc(0, 1000, out)  # 168 primes do not fit in 16 slots
        assert e.value.status == binding.ERR_CAPACITY
        # the widest range the header promises fits, at an unaligned start
        lo = 6 * 10**10 + 5
        n = sv.range_count(lo, lo + MAX_WIDTH_DEFAULT_TILE).count
        big = torch.empty(n + 8, dtype=torch.int64, device="cuda")
        got, cs = sv.range_list_noalloc(lo, lo + MAX_WIDTH_DEFAULT_TILE, big)
        assert got == n
        ref = sv.range_count(lo, lo + MAX_WIDTH_DEFAULT_TILE)
        assert (cs.count, cs.checksum) == (ref.count, ref.checksum)
        with pytest.raises(binding.SieveError):
            sv.range_list_noalloc(lo, lo + MAX_WIDTH_DEFAULT_TILE + 12, big)
