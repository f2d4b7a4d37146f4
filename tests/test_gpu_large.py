"""GPU parity at full size: the [2, 1e12] count with its 2^30-number block
histogram (checked against the published pi(1e12), against the oracle on
sampled blocks, and by additivity), and windows near 1e18 / 2^63 (checked
against Miller-Rabin on every integer and against the oracle)."""
import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_count_1e12_histogram():
    """Every one of the 932 bins and the checksum against the oracle's full
    run (tests/golden/count_1e12_bins.json, written by
    tests/golden/make_count_1e12_bins.py from the oracle alone and checked
    there against OEIS A006880 / A046731), plus sampled blocks against a live
    oracle run and additivity over two halves."""
    _need_gpu()
    g = C.golden("pi_powers_of_ten.json")
    full = C.golden("count_1e12_bins.json")
    wl = workloads.COUNT_1E12
    assert (full["lo"], full["hi_exclusive"], full["seg_width"]) == (wl.lo, wl.hi, wl.seg_width)
    with binding.Sieve(wl.hi) as sv:
        tot, bins = sv.segment_counts(wl.lo, wl.hi, wl.seg_width)
        assert len(bins) == 932
        assert tot.count == g["pi"]["12"] == full["count"]
        assert tot.checksum == full["checksum_mod_2_64"] == full["sum_below_1e12"] % 2**64
        np.testing.assert_array_equal(bins, np.array(full["bins"], dtype=np.uint64))
        # the count-only path (no bins) and the host-output path agree with it
        r = sv.range_count(wl.lo, wl.hi)
        assert (r.count, r.checksum) == (tot.count, tot.checksum)
        # additivity of the checksum over two halves
        mid = 6 * 10**11 + 12345
        a = sv.range_count(wl.lo, mid)
        b = sv.range_count(mid, wl.hi)
        assert a.count + b.count == tot.count
        assert (a.checksum + b.checksum) % 2**64 == tot.checksum
        # sampled blocks against a live oracle run (first, a middle one, two random, the partial last)
        base = oracle.base_table(10**6)
        rng = np.random.default_rng(12)
        picks = sorted({0, 465, len(bins) - 1} | {int(x) for x in rng.integers(1, len(bins) - 1, size=2)})
        for i in picks:
            lo = max(wl.lo, i * wl.seg_width)
            hi = min(wl.hi, (i + 1) * wl.seg_width)
            oc, osum = oracle.count_range(lo, hi, base=base)
            assert int(bins[i]) == oc, i
            r = sv.range_count(lo, hi)
            assert (r.count, r.checksum) == (oc, osum), i


def test_windows_near_2_63_miller_rabin():
    _need_gpu()
    with binding.Sieve(2**63) as sv:
        lim, n, _ = sv.base_table()
        assert lim == 3037000499
        for lo in (10**18 - 5000, 10**18 + 10**9 - 4000, 2**62 + 1, 2**63 - 20001):
            hi = min(lo + 20000, 2**63)
            got = sv.range_list(lo, hi).tolist()
            want = [x for x in range(lo, hi) if C.mr_is_prime(x)]
            assert got == want, lo
            r = sv.range_count(lo, hi)
            assert (r.count, r.checksum) == (len(want), sum(want) % 2**64), lo


def test_window_1e18_oracle():
    _need_gpu()
    lo, hi = 10**18, 10**18 + 300_000
    with binding.Sieve(10**18 + 10**9) as sv:
        base = oracle.base_table(10**9)
        want = oracle.list_range(lo, hi, base=base)
        got = sv.range_list(lo, hi)
        assert np.array_equal(got, want)


def test_far_range_routes_and_matches():
    """A range far up ([1e18, 1e18 + 2e7): 5e7 base primes) goes through the
    bucket sieve by default; with the bucket sieve off, sieve_range sends it to
    the batch path's strips (a one-query batch); and one segment-path launch
    with the bucket sieve off (range_batch(naive=True)) locates every prime in
    every tile.  All three must give the same counts and lists, equal to the
    oracle's."""
    _need_gpu()
    lo, hi = 10**18, 10**18 + 2 * 10**7
    with binding.Sieve(hi) as sv:
        sv.set_phase_timing(True)
        got = sv.range_count(lo, hi)
        assert sv.phase_times()["bucket_waves"] > 0
        lst = sv.range_list(lo, hi)
        sv.set_options(bucket_threshold=0)
        strips = sv.range_count(lo, hi)
        lst_s = sv.range_list(lo, hi)
        cnt_e, off_e, vals_e = sv.range_batch([lo], [hi], [1], naive=True)
    assert (got.count, got.checksum) == (strips.count, strips.checksum) == (int(cnt_e[0][0]), int(cnt_e[0][1]))
    np.testing.assert_array_equal(lst, vals_e)
    np.testing.assert_array_equal(lst_s, vals_e)
    want = oracle.count_range(lo, hi)
    assert (got.count, got.checksum) == want
    assert lst.size == want[0]
    for x in lst[:: max(1, lst.size // 64)].tolist():
        assert C.mr_is_prime(int(x))
