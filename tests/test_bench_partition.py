"""Host logic of bench.py's multi-GPU partition (no GPU): rank 0 keeps the
headline range [2, 1e12]; every other rank takes the next contiguous range
whose modelled count time equals rank 0's, so that per-GPU work is fixed."""
import bench


def test_rank_ranges_contiguous_and_balanced():
    r0 = bench.rank_range(0)
    assert r0 == (2, 10**12 + 1)
    target = bench.range_cost_ms(*r0)
    prev_hi, prev_w = r0[1], r0[1] - r0[0]
    for r in range(1, 8):
        lo, hi = bench.rank_range(r)
        assert lo == prev_hi and (hi - lo) % 6_000_000 == 0
        assert hi - lo < prev_w  # higher ranges cost more per number
        cost = bench.range_cost_ms(lo, hi)
        assert target - 0.01 * target <= cost <= target
        prev_hi, prev_w = hi, hi - lo


def test_cost_model_matches_its_measurements():
    # the windows the model was fitted to, in ms per 1e11 numbers
    for lo, ms in ((10**12, 18.60), (4 * 10**12, 22.96), (10**13, 27.86), (2 * 10**13, 33.26)):
        got = bench.range_cost_ms(lo, lo + 10**11)
        assert abs(got - ms) <= 0.02 * ms, (lo, got, ms)
