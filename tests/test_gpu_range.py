"""GPU parity: counts, checksums, per-segment counts and lists of the CUDA
path against the CPU oracle, bit-exact (integer results; no tolerance)."""
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
    s = binding.Sieve(10**13)
    yield s
    s.close()


def _oracle_base(hi):
    return oracle.base_table(max(oracle.isqrt(max(hi, 2) - 1), 100))


EDGE_RANGES = [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 3), (3, 4), (2, 4), (4, 5), (5, 6),
               (0, 6), (0, 7), (1, 8), (5, 25), (0, 26), (24, 26), (25, 26), (6, 7), (7, 8),
               (0, 100), (10, 30), (19, 24), (23, 24), (0, 530), (528, 530), (529, 530), (0, 1000)]


def test_edge_ranges_count_and_list(sv):
    for lo, hi in EDGE_RANGES:
        want = C.brute_primes(lo, hi)
        r = sv.range_count(lo, hi)
        assert (r.count, r.checksum) == (len(want), sum(want) % 2**64), (lo, hi)
        got = sv.range_list(lo, hi).tolist() if want else []
        assert got == want, (lo, hi)


def test_random_small_ranges(sv):
    q = workloads.random_small_ranges(300, seed=17, max_lo=10**7, max_width=200_000)
    for lo, hi in zip(q.lo.tolist(), q.hi.tolist()):
        want = oracle.count_range(lo, hi)
        r = sv.range_count(lo, hi)
        assert (r.count, r.checksum) == want, (lo, hi)


def test_prime_square_boundaries(sv):
    """Ranges that start or end at p^2, p^2 + 1 for base primes p (first strikes)."""
    for p in (23, 29, 31, 97, 101, 1009, 7919, 65521, 99991, 999983):
        cases = [(p * p, p * p + 1), (p * p - 1, p * p + 2), (p * p - 100, p * p), (max(0, p * p - 6001), p * p + 7001)]
        if p < 5000:
            cases.append((p, p * p + 1000))
        for lo, hi in cases:
            want = oracle.count_range(lo, hi, base=_oracle_base(hi))
            r = sv.range_count(lo, hi)
            assert (r.count, r.checksum) == want, (p, lo, hi)


def test_lists_against_oracle(sv):
    for lo, hi in ((0, 10**6), (999_000, 2_345_678), (10**9, 10**9 + 3_000_001), (2**33 + 7, 2**33 + 1_500_000)):
        want = oracle.list_range(lo, hi, base=_oracle_base(hi))
        got = sv.range_list(lo, hi)
        assert got.dtype == np.uint64
        assert np.array_equal(got, want), (lo, hi)


def test_primes_u32_1e8(sv):
    """[2, 1e8] as a uint32 list: pi = 5761455, sum = 279209790387276, equal to the oracle."""
    g = C.golden("pi_powers_of_ten.json")
    out = np.zeros(5_800_000, dtype=np.uint32)
    n = sv.primes(10**8, out)
    assert n == g["pi"]["8"]
    got = out[:n]
    assert int(got.astype(np.uint64).sum()) == g["sum_below"]["8"]
    want = oracle.list_range(2, 10**8 + 1).astype(np.uint32)
    assert np.array_equal(got, want)
    r = sv.count(10**8)
    assert (r.count, r.checksum) == (g["pi"]["8"], g["sum_below"]["8"])


def test_published_counts(sv):
    g = C.golden("pi_powers_of_ten.json")
    for e in range(1, 11):
        r = sv.count(10**e)
        assert r.count == g["pi"][str(e)], e
        assert r.checksum == g["sum_below"][str(e)] % 2**64, e


def test_segment_counts_1e10(sv):
    """[2, 1e10] with 2^24-number segments: 597 bins, against the oracle."""
    wl = workloads.SEGMENTED_1E10
    tot, bins = sv.segment_counts(wl.lo, wl.hi, wl.seg_width)
    assert len(bins) == 597
    assert tot.count == 455052511 and int(bins.sum()) == tot.count
    oc, osum, obins = oracle.segment_counts(wl.lo, wl.hi, wl.seg_width)
    assert (tot.count, tot.checksum) == (oc, osum)
    assert np.array_equal(bins, obins)
    assert int(bins.max()) < 2**32  # the per-segment counts fit uint32


def test_segment_counts_odd_widths(sv):
    for lo, hi, w in ((0, 10**7, 6144), (12345, 9_876_543, 1_000_003), (10**11, 10**11 + 5 * 10**7, 1 << 23),
                      (7, 8, 10**6)):
        tot, bins = sv.segment_counts(lo, hi, w)
        oc, osum, obins = oracle.segment_counts(lo, hi, w, base=_oracle_base(hi))
        assert (tot.count, tot.checksum) == (oc, osum), (lo, hi, w)
        assert np.array_equal(bins, obins), (lo, hi, w)


@pytest.mark.parametrize("tile_bits", [1024, 4096, 32768, 1 << 18, 1 << 19])
@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_option_sweep(sv, tile_bits, threads):
    old = sv.options()
    try:
        sv.set_options(tile_bits=tile_bits, block_threads=threads, group_hits=1 + (threads // 256),
                       presieve_groups=(tile_bits.bit_length() + threads.bit_length()) % 9)
        for lo, hi in ((0, 3_000_000), (10**10 - 777, 10**10 + 4_000_000)):
            r = sv.range_count(lo, hi)
            assert (r.count, r.checksum) == oracle.count_range(lo, hi, base=_oracle_base(hi)), (lo, hi)
        lo, hi = 10**9 + 11, 10**9 + 700_000
        assert np.array_equal(sv.range_list(lo, hi), oracle.list_range(lo, hi))
    finally:
        sv.set_options(**old)


def test_device_outputs_and_async(sv):
    torch = pytest.importorskip("torch")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    sv.range_count(10**9, 2 * 10**9, out=out, asynchronous=True)
    torch.cuda.synchronize()
    want = oracle.count_range(10**9, 2 * 10**9)
    assert [int(x) % 2**64 for x in out.tolist()] == list(want)
    lo, hi, w = 2, 10**9 + 1, 1 << 24
    nb = binding.Sieve.nbins(lo, hi, w)
    cnt = torch.zeros(nb, dtype=torch.int64, device="cuda")
    tot = torch.zeros(2, dtype=torch.int64, device="cuda")
    sv.segment_counts(lo, hi, w, counts=cnt, total=tot)
    oc, osum, obins = oracle.segment_counts(lo, hi, w)
    assert int(tot[0]) == oc and int(tot[1]) % 2**64 == osum
    assert np.array_equal(cnt.cpu().numpy().astype(np.uint64), obins)
    lst = torch.zeros(60_000, dtype=torch.int64, device="cuda")
    n = sv.range_list(10**12, 10**12 + 1_000_000, out=lst)
    want = oracle.list_range(10**12, 10**12 + 1_000_000, base=_oracle_base(10**12 + 10**6))
    assert n == want.size
    assert np.array_equal(lst[:n].cpu().numpy().astype(np.uint64), want)


def test_errors(sv):
    with pytest.raises(binding.SieveError) as e:
        sv.range_count(10, 5)
    assert e.value.status == binding.ERR_INVALID
    with pytest.raises(binding.SieveError) as e:
        sv.range_count(0, 10**14)
    assert e.value.status == binding.ERR_RANGE
    out = np.zeros(10, dtype=np.uint64)
    with pytest.raises(binding.SieveError) as e:
        sv.range_list(0, 1000, out)
    assert e.value.status == binding.ERR_CAPACITY
    assert np.all(out == 0)  # nothing written when the list does not fit
    with pytest.raises(binding.SieveError):
        sv.segment_counts(0, 10**6, 100)  # width below the minimum
    with pytest.raises(binding.SieveError):
        sv.set_options(tile_bits=1000)
    with pytest.raises(binding.SieveError):
        sv.set_options(tile_bits=3 << 10)  # not a power of two
    with pytest.raises(binding.SieveError):
        sv.set_options(tile_bits=1 << 20)  # 256 KB of bitmaps do not fit in shared memory
    r = sv.range_count(77, 77)
    assert (r.count, r.checksum) == (0, 0)


def test_phase_timing(sv):
    """Per-phase CUDA-event timing of a range call: the tile kernel, scan and
    compaction times are positive in list mode, the listed count matches, and
    timing changes no result."""
    import torch

    lo, hi = 10**9, 10**9 + 3 * 10**7
    with binding.Sieve(hi) as sv:  # a context of its own: timing is off by default
        want = sv.range_count(lo, hi)
        with pytest.raises(binding.SieveError):
            sv.phase_times()
        sv.set_phase_timing(True)
        got = sv.range_count(lo, hi)
        t = sv.phase_times()
        assert (got.count, got.checksum) == (want.count, want.checksum)
        assert t["sieve_ms"] > 0 and t["scan_ms"] == 0 and t["compact_ms"] == 0 and t["listed"] == 0
        assert t["tiles"] * t["tile_len"] >= (hi - lo) // 6
        out = torch.zeros(want.count, dtype=torch.int64, device="cuda")
        n = sv.range_list(lo, hi, out=out)  # two passes (default): tile kernel, scan, compaction
        t = sv.phase_times()
        assert n == want.count == t["listed"]
        assert t["sieve_ms"] > 0 and t["scan_ms"] > 0 and t["compact_ms"] > 0
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), oracle.list_range(lo, hi))
        sv.set_options(list_single_pass=1)  # one pass: the tile kernel writes the list
        out.zero_()
        n = sv.range_list(lo, hi, out=out)
        t = sv.phase_times()
        assert n == want.count == t["listed"]
        assert t["sieve_ms"] > 0 and t["scan_ms"] == 0 and t["compact_ms"] == 0
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.uint64), oracle.list_range(lo, hi))
        sv.set_phase_timing(False)
        with pytest.raises(binding.SieveError):
            sv.phase_times()
