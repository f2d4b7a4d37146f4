"""GPU parity of the single-pass list path: lists written into device memory
by the tile kernel itself (each tile compacted from shared memory at an
offset found by decoupled look-back) against the CPU oracle and against the
two-pass path (bitmaps, scan, compaction), bit-exact (integer results): edge
and random ranges, uint32 and uint64 outputs, the capacity rule, and far
ranges whose large primes go through the bucket sieve."""
import numpy as np
import pytest

import oracle
from paper_2310_17746_gb300 import binding, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def sv(torch):
    s = binding.Sieve(10**15)
    s.set_phase_timing(True)
    s.set_options(list_single_pass=1)
    yield s
    s.close()


def _dev_list(sv, torch, lo, hi, single_pass=1, extra=16):
    n = sv.range_count(lo, hi).count
    out = torch.full((n + extra,), -1, dtype=torch.int64, device="cuda")
    old = sv.options()
    try:
        sv.set_options(list_single_pass=single_pass)
        got = sv.range_list(lo, hi, out=out)
        if single_pass:
            assert sv.phase_times()["compact_ms"] == 0.0  # the tile kernel wrote the list
    finally:
        sv.set_options(**old)
    assert got == n
    assert bool((out[n:] == -1).all()), (lo, hi)
    return out[:n].cpu().numpy().astype(np.uint64)


EDGES = [(0, 1), (0, 2), (0, 3), (0, 4), (2, 3), (3, 4), (0, 26), (24, 26), (25, 26), (0, 1000), (5, 25),
         (10**12 - 100, 10**12 + 100), (10**15 - 1000, 10**15)]


def test_single_pass_edges_and_random(sv, torch):
    q = workloads.random_small_ranges(60, seed=41, max_lo=10**14, max_width=3_000_000)
    for lo, hi in EDGES + list(zip(q.lo.tolist(), q.hi.tolist())):
        want = oracle.list_range(lo, hi)
        if want.size == 0:
            continue
        np.testing.assert_array_equal(_dev_list(sv, torch, lo, hi), want)


def test_single_pass_equals_two_pass_wide(sv, torch):
    for lo, hi in ((10**12, 10**12 + 2 * 10**9), (2, 3 * 10**9), (7 * 10**13 + 11, 7 * 10**13 + 3 * 10**9 + 11)):
        one = _dev_list(sv, torch, lo, hi, 1)
        two = _dev_list(sv, torch, lo, hi, 0)
        np.testing.assert_array_equal(one, two)
        a, b = int(one[0]), int(one[-1])
        assert a >= lo and b < hi and (np.diff(one) > 0).all()
    lo, hi = 10**12, 10**12 + 2 * 10**8
    np.testing.assert_array_equal(_dev_list(sv, torch, lo, hi), oracle.list_range(lo, hi))


def test_single_pass_uint32_primes(sv, torch):
    n = 5761455
    out = torch.full((n + 8,), -1, dtype=torch.int32, device="cuda")
    assert sv.primes(10**8, out=out) == n
    assert bool((out[n:] == -1).all())
    got = out[:n].cpu().numpy().astype(np.uint64)
    np.testing.assert_array_equal(got, oracle.list_range(0, 10**8 + 1))


def test_single_pass_capacity(sv, torch):
    lo, hi = 10**11, 10**11 + 10**8
    n = sv.range_count(lo, hi).count
    cap = n // 3
    out = torch.full((cap + 100,), -1, dtype=torch.int64, device="cuda")
    with pytest.raises(binding.SieveError) as e:
        sv.range_list(lo, hi, out=out[:cap])
    assert e.value.status == binding.ERR_CAPACITY
    assert bool((out[cap:] == -1).all()), "written past the capacity"


def test_single_pass_with_buckets(sv, torch):
    lo, hi = 10**15 - 2 * 10**9, 10**15  # a bitmap beyond L2: the bucket sieve, not the strips route
    got = _dev_list(sv, torch, lo, hi)
    assert sv.phase_times()["bucket_waves"] > 0
    np.testing.assert_array_equal(got, oracle.list_range(lo, hi))
