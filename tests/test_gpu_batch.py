"""GPU parity of the batched launch (sieve_range_batch): every query's count,
checksum and list against the CPU oracle, bit-exact (integer results, no
tolerance), and against the one-launch-per-query path (sieve_range_each).

The cases cover the two kinds of work items -- tile items sized to narrow
queries, and the strips that locate the primes above the tile length once per
query -- in both output modes, plus empty and ragged queries, capacity
handling and the tunables."""
import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

MAX_HI = 10**16


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = binding.Sieve(MAX_HI)
    yield s
    s.close()


_BASES = {}


def _base(hi):
    """Oracle base table covering isqrt(hi - 1), shared between queries."""
    s = oracle.isqrt(max(hi, 2) - 1)
    lim = 1024
    while lim < s:
        lim *= 2
    if lim not in _BASES:
        _BASES[lim] = oracle.BaseTable(lim)
    return _BASES[lim]


def _check_against_oracle(lo, hi, mode, cnt, offsets, values, idx=None):
    idx = range(len(lo)) if idx is None else idx
    for i in idx:
        a, b = int(lo[i]), int(hi[i])
        want = oracle.count_range(a, b, base=_base(b))
        got = (int(cnt[i][0]), int(cnt[i][1]))
        assert got == want, (i, a, b, got, want)
        run = values[int(offsets[i]):int(offsets[i + 1])]
        if mode[i] == workloads.MODE_LIST:
            assert run.size == want[0], (i, a, b)
            if want[0]:
                np.testing.assert_array_equal(run, oracle.list_range(a, b, base=_base(b)))
        else:
            assert run.size == 0, (i, a, b)


def _restore(sv, opts):
    sv.set_options(**opts)


EDGES = [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 3), (3, 4), (2, 4), (4, 5), (5, 6), (0, 6),
         (0, 7), (1, 8), (5, 25), (0, 26), (24, 26), (25, 26), (6, 7), (7, 8), (0, 100), (10, 30), (19, 24),
         (23, 24), (0, 530), (528, 530), (529, 530), (0, 1000), (7, 7), (10**12, 10**12),
         (10**15 - 1, 10**15 + 1), (2**53 - 1000, 2**53 + 1000)]


def test_batch_edges_both_modes(sv):
    lo = np.array([a for a, _ in EDGES] * 2, dtype=np.uint64)
    hi = np.array([b for _, b in EDGES] * 2, dtype=np.uint64)
    mode = np.array([0] * len(EDGES) + [1] * len(EDGES), dtype=np.uint8)
    cnt, off, vals = sv.range_batch(lo, hi, mode)
    for i in range(lo.size):
        a, b = int(lo[i]), int(hi[i])
        want = C.brute_primes(a, b) if b < 10**7 else oracle.list_range(a, b, base=_base(b)).tolist()
        assert (int(cnt[i][0]), int(cnt[i][1])) == (len(want), sum(want) % 2**64), (a, b)
        run = vals[int(off[i]):int(off[i + 1])].tolist()
        assert run == (want if mode[i] else []), (a, b)


def test_batch_empty_and_single(sv):
    cnt, off, vals = sv.range_batch(np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0, np.uint8))
    assert cnt.shape == (0, 2) and off.tolist() == [0] and vals.size == 0
    cnt, off, vals = sv.range_batch([10**9], [10**9 + 10**6], [1])
    np.testing.assert_array_equal(vals, oracle.list_range(10**9, 10**9 + 10**6))


def test_batch_random_small(sv):
    q = workloads.random_small_ranges(400, seed=5, max_lo=10**9, max_width=300_000)
    cnt, off, vals = sv.range_batch(q.lo, q.hi, q.mode)
    _check_against_oracle(q.lo, q.hi, q.mode, cnt, off, vals)


def _high_queries():
    lo, hi, mode = [], [], []
    for base in (10**12, 10**13 + 12345, 10**14, 10**15 - 7, 10**16 - 4 * 10**6):
        for w in (1, 6, 1000, 65_537, 1_000_003, 3_000_000):
            for m in (0, 1):
                lo.append(base)
                hi.append(base + w)
                mode.append(m)
    return (np.array(lo, dtype=np.uint64), np.array(hi, dtype=np.uint64), np.array(mode, dtype=np.uint8))


def test_batch_high_queries_strips(sv):
    """High, narrow-to-medium queries: most are merged (strips over many base primes)."""
    lo, hi, mode = _high_queries()
    cnt, off, vals = sv.range_batch(lo, hi, mode)
    _check_against_oracle(lo, hi, mode, cnt, off, vals)


@pytest.mark.parametrize("tile_bits,threads,chunk", [(1 << 12, 256, 1024), (1 << 14, 512, 4096),
                                                     (1 << 16, 1024, 1 << 15), (1 << 19, 1024, 1 << 17)])
def test_batch_tunables_same_result(sv, tile_bits, threads, chunk):
    """Small tiles and small strips force multi-tile merged queries; every
    setting must give the oracle's answer."""
    opts = sv.options()
    try:
        sv.set_options(batch_tile_bits=tile_bits, block_threads=threads, chunk_primes=chunk)
        lo, hi, mode = _high_queries()
        q = workloads.random_small_ranges(60, seed=11, max_lo=10**11, max_width=2_000_000)
        lo = np.concatenate([lo, q.lo])
        hi = np.concatenate([hi, q.hi])
        mode = np.concatenate([mode, q.mode])
        cnt, off, vals = sv.range_batch(lo, hi, mode)
        _check_against_oracle(lo, hi, mode, cnt, off, vals)
    finally:
        _restore(sv, opts)


def test_batch_workload_vs_each_and_oracle(sv):
    """The 4096-query batch workload (seed 0): the batched launch equals the
    one-launch-per-query path on every query, and the oracle on a sample."""
    torch = pytest.importorskip("torch")
    q = workloads.batch_queries()
    nq = len(q)
    cnt_b = torch.zeros((nq, 2), dtype=torch.int64, device="cuda")
    off_b = torch.zeros(nq + 1, dtype=torch.int64, device="cuda")
    # size the list output from a count-only pass of the same batch
    cnt0, _, _ = sv.range_batch(q.lo, q.hi, np.zeros(nq, np.uint8))
    need = int(sum(int(cnt0[i][0]) for i in range(nq) if q.mode[i]))
    vals_b = torch.empty(max(need, 1), dtype=torch.int64, device="cuda")
    total = sv.range_batch(q.lo, q.hi, q.mode, cnt=cnt_b, offsets=off_b, values=vals_b)
    assert total == need
    cnt_e, off_e, vals_e = sv.range_batch(q.lo, q.hi, q.mode, naive=True)
    np.testing.assert_array_equal(cnt_b.cpu().numpy().astype(np.uint64), cnt_e)
    np.testing.assert_array_equal(off_b.cpu().numpy().astype(np.uint64), off_e)
    np.testing.assert_array_equal(vals_b[:total].cpu().numpy().astype(np.uint64), vals_e)
    np.testing.assert_array_equal(cnt0, cnt_e)  # count-only and list runs agree
    # oracle on a seeded sample of the queries (bounded oracle time)
    rng = np.random.default_rng(123)
    width = (q.hi - q.lo).astype(np.int64)
    pool = np.nonzero(width <= 3_000_000)[0]
    sample = rng.choice(pool, size=48, replace=False)
    _check_against_oracle(q.lo, q.hi, q.mode, cnt_e, off_e, vals_e, idx=sample.tolist())


def test_batch_capacity(sv):
    lo = np.array([10**6, 10**9, 10**12], dtype=np.uint64)
    hi = lo + np.array([10**5, 10**5, 10**5], dtype=np.uint64)
    mode = np.ones(3, dtype=np.uint8)
    cnt, off, vals = sv.range_batch(lo, hi, mode)
    need = int(off[-1])
    small = np.zeros(need - 1, dtype=np.uint64)
    with pytest.raises(binding.SieveError) as e:
        sv.range_batch(lo, hi, mode, values=small)
    assert e.value.status == binding.ERR_CAPACITY
    # the exact size works, host and device
    cnt2, off2, vals2 = sv.range_batch(lo, hi, mode, values=np.zeros(need, dtype=np.uint64))
    np.testing.assert_array_equal(vals2, vals)


def test_batch_host_device_agree(sv):
    torch = pytest.importorskip("torch")
    q = workloads.random_small_ranges(200, seed=9, max_lo=10**13, max_width=500_000)
    cnt, off, vals = sv.range_batch(q.lo, q.hi, q.mode)
    c = torch.zeros((len(q), 2), dtype=torch.int64, device="cuda")
    o = torch.zeros(len(q) + 1, dtype=torch.int64, device="cuda")
    v = torch.zeros(max(vals.size, 1), dtype=torch.int64, device="cuda")
    n = sv.range_batch(q.lo, q.hi, q.mode, cnt=c, offsets=o, values=v)
    assert n == vals.size
    np.testing.assert_array_equal(c.cpu().numpy().astype(np.uint64), cnt)
    np.testing.assert_array_equal(o.cpu().numpy().astype(np.uint64), off)
    np.testing.assert_array_equal(v[:n].cpu().numpy().astype(np.uint64), vals)


def test_batch_rejects_bad_queries(sv):
    for lo, hi, mode, status in (([5], [4], [0], binding.ERR_INVALID), ([0], [10], [2], binding.ERR_INVALID),
                                 ([0], [MAX_HI * 2], [0], binding.ERR_RANGE)):
        with pytest.raises(binding.SieveError) as e:
            sv.range_batch(lo, hi, mode)
        assert e.value.status == status
    # the context still works afterwards
    cnt, _, _ = sv.range_batch([0], [100], [0])
    assert int(cnt[0][0]) == 25


def test_batch_single_huge_tile_is_split(sv):
    """A lone narrow query high up has one tile with millions of base primes:
    the planner splits that tile's primes over many items (shared-memory
    pieces ANDed in global memory)."""
    for lo, hi, m in ((10**16 - 1000, 10**16, 1), (10**16 - 5 * 10**6, 10**16 - 4 * 10**6, 0)):
        cnt, off, vals = sv.range_batch([lo], [hi], [m])
        _check_against_oracle(np.array([lo], np.uint64), np.array([hi], np.uint64), np.array([m], np.uint8),
                              cnt, off, vals)


def test_batch_strip_primes_squared_inside_queries(sv):
    """Queries centred on P^2 for primes P far above the break-even prime of
    the strips (small batch tiles): such a strip prime starts at its square
    (the clamp path of the start computation), the others from the inverse of
    6.  Both modes, against the oracle."""
    opts = sv.options()
    try:
        sv.set_options(batch_tile_bits=1 << 12, block_threads=512, chunk_primes=1024)
        lo, hi, mode = [], [], []
        for near in (10**6, 2 * 10**6, 3_162_000):
            p = int(oracle.list_range(near, near + 200)[0])
            sq = p * p
            for half in (60_000, 300_000):
                for m in (0, 1):
                    lo.append(sq - half)
                    hi.append(sq + half + 1)
                    mode.append(m)
            lo.append(sq)  # the square is the query's first value
            hi.append(sq + 200_000)
            mode.append(1)
        lo = np.array(lo, dtype=np.uint64)
        hi = np.array(hi, dtype=np.uint64)
        mode = np.array(mode, dtype=np.uint8)
        cnt, off, vals = sv.range_batch(lo, hi, mode)
        _check_against_oracle(lo, hi, mode, cnt, off, vals)
    finally:
        _restore(sv, opts)


def test_batch_phase_times(sv):
    """With phase timing on, a batch call reports its host planning time and
    its graph's device time; the results are unchanged."""
    q = workloads.random_small_ranges(300, seed=11, max_lo=10**12, max_width=2_000_000)
    cnt0, off0, vals0 = sv.range_batch(q.lo, q.hi, q.mode)
    sv.set_phase_timing(True)
    try:
        cnt, off, vals = sv.range_batch(q.lo, q.hi, q.mode)
        ph = sv.phase_times()
    finally:
        sv.set_phase_timing(False)
    assert ph["batch_plan_ms"] > 0 and ph["sieve_ms"] > 0
    np.testing.assert_array_equal(cnt, cnt0)
    np.testing.assert_array_equal(off, off0)
    np.testing.assert_array_equal(vals, vals0)
    _check_against_oracle(q.lo, q.hi, q.mode, cnt, off, vals)
