"""GPU tests of the serving loop (sieve_server_*): every answer equals the
CPU oracle's and is the same whether the request ran alone or in a mix of
concurrent requests (bit-exact: integer results, no tolerance); admission by
device memory (backpressure), collection errors, and batches that overlap."""
import time

import numpy as np
import pytest

import oracle
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


def _collect(srv, ids, timeout_s=120.0):
    """Results of every id, collected in completion order."""
    out = {}
    pending = set(ids)
    t_end = time.time() + timeout_s
    while pending:
        assert time.time() < t_end, f"{len(pending)} requests not finished"
        rid = srv.next_done(timeout_us=100_000)
        if rid is None or rid not in pending:
            continue
        res = srv.poll(rid)
        assert res is not None
        out[rid] = res
        pending.discard(rid)
    return out


def _mix():
    q = workloads.random_small_ranges(150, seed=21, max_lo=10**12, max_width=400_000)
    lo, hi, mode = q.lo.tolist(), q.hi.tolist(), q.mode.tolist()
    for base in (10**13, 10**14 + 77, 10**15, 10**16 - 2 * 10**6):
        for w, m in ((1000, 0), (1000, 1), (250_000, 0), (250_000, 1), (2_000_000, 1)):
            lo.append(base)
            hi.append(base + w)
            mode.append(m)
    return lo, hi, mode


def _same(a, b):
    (ca, la), (cb, lb) = a, b
    assert (ca.count, ca.checksum) == (cb.count, cb.checksum)
    if la is None or lb is None:
        assert la is None and lb is None
    else:
        np.testing.assert_array_equal(la, lb)


def test_server_mix_equals_alone_and_oracle(sv):
    lo, hi, mode = _mix()
    with binding.Server(sv, pool_bytes=1 << 30) as srv:
        ids = [srv.submit(a, b, m) for a, b, m in zip(lo, hi, mode)]
        mixed = _collect(srv, ids)
        alone = []
        for a, b, m in zip(lo, hi, mode):
            rid = srv.submit(a, b, m)
            alone.append(_collect(srv, [rid])[rid])
        st = srv.stats()
    assert st["completed"] == 2 * len(lo)
    for i, rid in enumerate(ids):
        _same(mixed[rid], alone[i])
    base = oracle.BaseTable(10**8)
    for i, rid in enumerate(ids):
        c, lst = mixed[rid]
        want = oracle.count_range(lo[i], hi[i], base=base)
        assert (c.count, c.checksum) == want, (lo[i], hi[i])
        if mode[i] == workloads.MODE_LIST and want[0]:
            np.testing.assert_array_equal(lst, oracle.list_range(lo[i], hi[i], base=base))
        elif mode[i] == workloads.MODE_LIST:
            assert lst is None


def test_server_backpressure_by_device_memory(sv):
    # a 4 MiB pool: 524288 primes of room, one list of width 2e6 (bound 275761)
    with binding.Server(sv, pool_bytes=4 << 20) as srv:
        with pytest.raises(binding.SieveError) as e:
            srv.submit(10**9, 10**9 + 10**8, workloads.MODE_LIST)  # could never fit
        assert e.value.status == binding.ERR_CAPACITY
        held = []
        while True:
            rid = srv.try_submit(10**9, 10**9 + 2_000_000, workloads.MODE_LIST)
            if rid is None:
                break
            held.append(rid)
            assert len(held) < 100
        assert held, "the first list request must be admitted"
        assert srv.stats()["rejected"] >= 1
        # count requests need no pool room
        cid = srv.submit(10**9, 10**9 + 2_000_000, workloads.MODE_COUNT)
        res = _collect(srv, held + [cid])
        # collected results released the pool: admission works again
        rid = srv.submit(10**9, 10**9 + 2_000_000, workloads.MODE_LIST)
        again = _collect(srv, [rid])[rid]
        _same(again, res[held[0]])
        assert srv.stats()["pool_used_bytes"] == 0
    want = oracle.list_range(10**9, 10**9 + 2_000_000)
    np.testing.assert_array_equal(res[held[0]][1], want)
    assert res[cid][0].count == want.size


def test_server_poll_capacity_and_errors(sv):
    with binding.Server(sv, pool_bytes=64 << 20) as srv:
        rid = srv.submit(10**10, 10**10 + 100_000, workloads.MODE_LIST)
        while srv.next_done(timeout_us=100_000) != rid:
            pass
        small = np.zeros(10, dtype=np.uint64)
        with pytest.raises(binding.SieveError) as e:
            srv.poll(rid, out=small)
        assert e.value.status == binding.ERR_CAPACITY
        c, lst = srv.poll(rid)  # still there; now collected
        np.testing.assert_array_equal(lst, oracle.list_range(10**10, 10**10 + 100_000))
        with pytest.raises(binding.SieveError) as e:
            srv.poll(rid)
        assert e.value.status == binding.ERR_NOT_FOUND
        for lo, hi, m, st in ((5, 4, 0, binding.ERR_INVALID), (0, 10, 3, binding.ERR_INVALID),
                              (0, 4 * MAX_HI, 0, binding.ERR_RANGE)):
            with pytest.raises(binding.SieveError) as e:
                srv.submit(lo, hi, m)
            assert e.value.status == st
        # empty ranges are answered too
        rid = srv.submit(100, 100, workloads.MODE_LIST)
        (c, lst), = _collect(srv, [rid]).values()
        assert c.count == 0 and lst is None


def test_server_overlaps_batches(sv):
    """A request that arrives while a long batch is on the GPU is launched on
    the other stream at once and finishes first."""
    with binding.Server(sv, pool_bytes=64 << 20) as srv:
        heavy = srv.submit(10**15, 10**15 + 3 * 10**9, workloads.MODE_COUNT)
        t0 = time.time()
        while srv.stats()["batches"] < 1:
            assert time.time() - t0 < 30
            time.sleep(0.0005)
        small = [srv.submit(10**12 + 1000 * i, 10**12 + 1000 * i + 5000, workloads.MODE_COUNT) for i in range(8)]
        order, t_done = [], {}
        pending = set(small + [heavy])
        while pending:
            rid = srv.next_done(timeout_us=1_000_000)
            if rid is not None:
                order.append(rid)
                t_done[rid] = time.time() - t0
                pending.discard(rid)
        st = srv.stats()
        res = {rid: srv.poll(rid) for rid in order}
    assert st["overlapped_batches"] >= 1
    assert order[-1] == heavy, ("the short requests must not wait for the long batch", t_done, heavy, st)
    want = oracle.count_range(10**15, 10**15 + 3 * 10**9)
    assert (res[heavy][0].count, res[heavy][0].checksum) == want
