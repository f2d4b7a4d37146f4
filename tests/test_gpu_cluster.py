"""GPU parity of cluster segments (cluster.cuh): C CTAs of a thread-block
cluster sieve C consecutive tiles together, the base primes above
cluster_threshold x L located once per segment and struck into the members'
shared memory through distributed shared memory.  Counts, checksums,
per-segment counts and lists against the CPU oracle (bit-exact: integer
results) for every cluster size and several thresholds, with segments whose
last members have no tile, tiles shrunk for short ranges, prime squares inside
the range, and against the default route at a larger size."""
import numpy as np
import pytest

import oracle
from paper_2310_17746_gb300 import binding

pytestmark = pytest.mark.gpu

MAX_HI = 10**15
SIZES = (2, 4, 8, 16)


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


def _with(sv, fn, **opts):
    old = sv.options()
    try:
        sv.set_options(**opts)
        return fn()
    finally:
        sv.set_options(**old)


def _count(sv, lo, hi, C, thr):
    def run():
        r = sv.range_count(lo, hi)
        return (r.count, r.checksum), sv.phase_times()
    return _with(sv, run, cluster_ctas=C, cluster_threshold=thr)


@pytest.mark.parametrize("C", SIZES)
@pytest.mark.parametrize("thr", [0, 4, 16])
def test_cluster_counts_equal_oracle(sv, base, C, thr):
    # 318 tiles of 2^19 indices: not a multiple of 4, 8 or 16 (the last
    # segment has members without a tile)
    lo, hi = 10**14 + 12345, 10**14 + 12345 + 10**9
    got, ph = _count(sv, lo, hi, C, thr)
    assert ph["cluster_ctas"] == C and ph["bucket_waves"] == 0
    assert got == oracle.count_range(lo, hi, base=base)


@pytest.mark.parametrize("C", [2, 8])
def test_cluster_odd_tile_count(sv, base, C):
    lo = 7 * 10**13 + 1
    hi = lo + 6 * (1 << 19) * 301 - 17  # 301 tiles: the last segment is ragged for C = 2 too
    got, ph = _count(sv, lo, hi, C, 0)
    assert ph["cluster_ctas"] == C and ph["tiles"] % C != 0
    assert got == oracle.count_range(lo, hi, base=base)


@pytest.mark.parametrize("C", [4, 16])
def test_cluster_all_lane_primes_near_start(sv, base, C):
    """Threshold 0 from the start of the numbers: every one-lane prime goes
    through the cluster strikes, with the P^2 clamp inside the first
    segments, 2 and 3, and the presieved primes' fix-ups."""
    for lo, hi in ((2, 10**9 + 1), (0, 123456789), (5, 6), (2, 3), (10**6, 10**6)):
        got, ph = _count(sv, lo, hi, C, 0)
        assert got == oracle.count_range(lo, hi, base=base), (lo, hi)
    assert _count(sv, 2, 10**9 + 1, C, 0)[0][0] == 50847534


@pytest.mark.parametrize("C", [2, 8])
def test_cluster_short_ranges_shrunk_tiles(sv, base, C):
    """Ranges shorter than one full tile per CTA slot get smaller tiles (down
    to 1024 indices), so a segment spans only a few thousand indices."""
    for lo, hi in ((10**12, 10**12 + 10**6), (10**14 - 5000, 10**14 + 5000), (999999999989, 1000000000039)):
        got, ph = _count(sv, lo, hi, C, 0)
        assert got == oracle.count_range(lo, hi, base=base), (lo, hi)


def test_cluster_across_prime_squares(sv, base):
    """Around the square of the largest base primes: their first hits are
    clamped at P^2 inside the segment."""
    p = 31622743  # the largest prime below sqrt(1e15)
    lo, hi = p * p - 3 * 10**8, min(p * p + 2 * 10**8, MAX_HI)
    for C, thr in ((4, 16), (8, 0)):
        got, _ = _count(sv, lo, hi, C, thr)
        assert got == oracle.count_range(lo, hi, base=base)


@pytest.mark.parametrize("C", [2, 8])
def test_cluster_segment_counts(sv, base, C):
    lo, hi, w = 10**14 + 12345, 10**14 + 12345 + 6 * 10**8, 1 << 26

    def run():
        return sv.segment_counts(lo, hi, w), sv.phase_times()
    (tot, bins), ph = _with(sv, run, cluster_ctas=C, cluster_threshold=4)
    assert ph["cluster_ctas"] == C
    oc, osum, obins = oracle.segment_counts(lo, hi, w, base=base)
    assert (tot.count, tot.checksum) == (oc, osum)
    np.testing.assert_array_equal(bins, obins)


@pytest.mark.parametrize("C", [4, 16])
def test_cluster_list_equals_oracle(sv, base, C):
    torch = pytest.importorskip("torch")
    lo, hi = 10**13 - 10**7 + 3, 10**13 + 2 * 10**7
    want = oracle.list_range(lo, hi, base=base)

    def run():
        out = torch.zeros(len(want) + 16, dtype=torch.int64, device="cuda")
        n = sv.range_list(lo, hi, out=out)
        return out[:n].cpu().numpy().astype(np.uint64), sv.phase_times()
    vals, ph = _with(sv, run, cluster_ctas=C, cluster_threshold=0)
    assert ph["cluster_ctas"] == C
    np.testing.assert_array_equal(vals, want)


def test_cluster_host_list(sv, base):
    lo, hi = 10**14 + 999, 10**14 + 999 + 3 * 10**7

    def run():
        return sv.range_list(lo, hi), sv.phase_times()
    vals, ph = _with(sv, run, cluster_ctas=8, cluster_threshold=4)
    assert ph["cluster_ctas"] == 8
    np.testing.assert_array_equal(vals, oracle.list_range(lo, hi, base=base))


def test_cluster_equals_default_route_far_up(sv):
    lo, hi = 10**15 - 2 * 10**10, 10**15
    default = sv.range_count(lo, hi)
    assert sv.phase_times()["cluster_ctas"] == 0
    for C, thr in ((8, 16), (16, 4)):
        got, ph = _count(sv, lo, hi, C, thr)
        assert ph["cluster_ctas"] == C
        assert got == (default.count, default.checksum)


def test_cluster_options_checked(sv):
    for bad in ({"cluster_ctas": 3}, {"cluster_ctas": 32}, {"cluster_threshold": 1025}):
        with pytest.raises(binding.SieveError):
            sv.set_options(**bad)
    assert sv.options()["cluster_ctas"] == 0
