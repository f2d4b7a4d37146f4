"""GPU parity of the bucket sieve for base primes far above the tile length
(bucket.cuh): ranges far up whose large primes are located once per wave of
tiles and whose hits reach the tiles through buckets.  Counts, checksums,
per-segment counts and lists against the CPU oracle and against the same
ranges with the bucket sieve switched off (bit-exact: integer results), for
several thresholds and wave sizes, across prime squares inside the range, and
with sub-buckets forced to overflow (the tiles' fallback)."""
import os

import numpy as np
import pytest

import oracle
from paper_2310_17746_gb300 import binding

pytestmark = pytest.mark.gpu

MAX_HI = 10**15


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = binding.Sieve(MAX_HI)
    s.set_phase_timing(True)
    yield s
    s.close()


@pytest.fixture(scope="module")
def base():
    return oracle.base_table(oracle.isqrt(MAX_HI - 1))


def _counts(sv, lo, hi, w, **opts):
    old = sv.options()
    try:
        sv.set_options(**opts)
        tot, bins = sv.segment_counts(lo, hi, w)
        waves = sv.phase_times()["bucket_waves"]
    finally:
        sv.set_options(**old)
    return (tot.count, tot.checksum), bins.copy(), waves


def test_bucket_counts_equal_oracle_and_plain(sv, base):
    lo, hi, w = 10**14 + 12345, 10**14 + 12345 + 2 * 10**9, 1 << 28
    got, bins, waves = _counts(sv, lo, hi, w)
    assert waves > 0, "the bucket sieve was not used"
    plain, pbins, pwaves = _counts(sv, lo, hi, w, bucket_threshold=0)
    assert pwaves == 0
    assert got == plain
    np.testing.assert_array_equal(bins, pbins)
    oc, osum, obins = oracle.segment_counts(lo, hi, w, base=base)
    assert got == (oc, osum)
    np.testing.assert_array_equal(bins, obins)


@pytest.mark.parametrize("threshold,wave,scatter", [(1, 1, 1), (2, 2, 2), (4, 1, 0), (8, 3, 2), (4, 4, 1)])
def test_bucket_tunables_same_result(sv, base, threshold, wave, scatter):
    lo, hi = 3 * 10**14 - 7, 3 * 10**14 - 7 + 6 * 10**8
    got, _, waves = _counts(sv, lo, hi, 1 << 30, bucket_threshold=threshold, bucket_wave=wave,
                            bucket_scatter=scatter)
    assert waves > 0
    assert got == oracle.count_range(lo, hi, base=base)


def test_bucket_list_across_prime_squares(sv, base):
    """A range around the square of the largest base primes: their first hits
    are clamped at P^2 inside the range.  One segment-path launch per query
    (range_batch(naive=True)) lists it through the bucket sieve."""
    p = 31622743  # the largest prime below sqrt(1e15)
    lo, hi = p * p - 3 * 10**8, min(p * p + 2 * 10**8, MAX_HI)
    cnt, off, vals = sv.range_batch([lo], [hi], [binding.LIST], naive=True)
    assert sv.phase_times()["bucket_waves"] > 0
    want = oracle.list_range(lo, hi, base=base)
    np.testing.assert_array_equal(vals, want)
    assert (int(cnt[0][0]), int(cnt[0][1])) == oracle.count_range(lo, hi, base=base)


@pytest.mark.parametrize("scatter", [1, 2])
def test_bucket_overflow_falls_back(sv, base, scatter):
    """Sub-buckets far too small (SIEVE_BUCKET_CAP): every tile finds its
    buckets overflowed and locates the large primes itself; same answer."""
    lo, hi = 10**14 + 5, 10**14 + 5 + 4 * 10**8
    os.environ["SIEVE_BUCKET_CAP"] = "32"
    try:
        small, sbins, waves = _counts(sv, lo, hi, 1 << 26, bucket_scatter=scatter)
    finally:
        del os.environ["SIEVE_BUCKET_CAP"]
    assert waves > 0
    full, fbins, _ = _counts(sv, lo, hi, 1 << 26, bucket_scatter=scatter)
    assert small == full == oracle.count_range(lo, hi, base=base)
    np.testing.assert_array_equal(sbins, fbins)


def test_far_ranges_route_to_buckets(sv, base):
    """sieve_range keeps a far range whose bitmap would not fit in L2 on the
    tile path when the bucket sieve applies (instead of the batch path's
    strips); both routes agree with the oracle."""
    lo, hi = 10**15 - 3 * 10**9, 10**15
    r = sv.range_count(lo, hi)
    assert sv.phase_times()["bucket_waves"] > 0
    old = sv.options()
    try:
        sv.set_options(bucket_threshold=0)
        s = sv.range_count(lo, hi)
    finally:
        sv.set_options(**old)
    assert (r.count, r.checksum) == (s.count, s.checksum) == oracle.count_range(lo, hi, base=base)
