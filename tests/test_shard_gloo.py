"""The multi-rank path on CPU: a range sharded over world_size 2 and 3 gloo
ranks (processes), each sieving its shard with the oracle, reduced with
torch.distributed, must equal the unsharded oracle result exactly (count,
checksum mod 2^64, per-segment counts, and the concatenated list)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2310_17746_gb300 import shard

LO, HI, W = 3, 6_000_011, 1 << 20
LLO, LHI = 10**9 - 100_000, 10**9 + 150_001


def test_shard_bounds_cover_in_order():
    for lo, hi, world in ((0, 100, 3), (5, 6, 4), (10**12, 10**12 + 10**7, 8), (7, 7, 2)):
        b = shard.shard_bounds(lo, hi, world)
        assert len(b) == world + 1 and b[0] == lo and b[-1] == hi
        assert all(x <= y for x, y in zip(b, b[1:]))
        assert all(x % 6 == 0 for x in b[1:-1] if lo < x < hi)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, s, bins = shard.distributed_segment_counts(lambda a, b, w: oracle.segment_counts(a, b, w), LO, HI, W)
        lst = shard.distributed_list(lambda a, b: oracle.list_range(a, b), LLO, LHI)
        out.put((rank, c, s, bins.tobytes(), lst.tobytes()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_equals_unsharded(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp

    ctx = tmp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_c, want_s, want_bins = oracle.segment_counts(LO, HI, W)
    want_list = oracle.list_range(LLO, LHI)
    for rank, c, s, bins, lst in res:
        assert (c, s) == (want_c, want_s), rank
        np.testing.assert_array_equal(np.frombuffer(bins, dtype=np.uint64), want_bins)
        np.testing.assert_array_equal(np.frombuffer(lst, dtype=np.uint64), want_list)


def test_shard_bounds_balance_modelled_cost():
    lo, hi = 2, 8 * 10**12
    b = shard.shard_bounds(lo, hi, 8)
    costs = [shard.cost_ms(x, y) for x, y in zip(b, b[1:])]
    assert max(costs) - min(costs) <= 0.002 * max(costs)
    widths = [y - x for x, y in zip(b, b[1:])]
    assert all(w1 > w2 for w1, w2 in zip(widths, widths[1:]))  # higher shards are narrower
    even = shard.shard_bounds(lo, hi, 8, balance=False)
    assert max(y - x for x, y in zip(even, even[1:])) - min(y - x for x, y in zip(even, even[1:])) <= 12
