"""The serving loop on its own workload: a seeded sample of the Poisson
request stream (seed 1: lo = floor(10^U(6, 18)), width = floor(10^U(3, 9)),
list mode with probability 0.2) against a context whose base table holds
every prime <= 1e9 (max_hi = 1e18 + 1e9), as the server is benchmarked.

Every answer is bit-exact (integer results, no tolerance):
  * the same in the concurrent mix and alone;
  * equal to the CPU oracle's count, checksum and list wherever the oracle
    finishes quickly (width <= 1e6);
  * for wider requests, equal to the regular single-range path (sieve_range:
    its own launches, outside the server), with Miller-Rabin on a stride of
    the listed primes and the list strictly increasing inside [lo, hi)."""
import time

import numpy as np
import pytest

import oracle
import oracle_checks as C
from paper_2310_17746_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

MAX_HI = 10**18 + 10**9 + 1
N_REQUESTS = 48
ORACLE_MAX_WIDTH = 10**6


def _collect(srv, ids, timeout_s=300.0):
    out, pending = {}, set(ids)
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


def test_serving_workload_sample_mix_alone_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    arr = workloads.serving_arrivals(10000.0, N_REQUESTS, seed=1)
    lo = [int(x) for x in arr.queries.lo]
    hi = [int(x) for x in arr.queries.hi]
    mode = [int(x) for x in arr.queries.mode]
    assert max(hi) <= MAX_HI and any(m == workloads.MODE_LIST for m in mode)
    with binding.Sieve(MAX_HI) as sv:
        lim, _, _ = sv.base_table()
        assert lim >= 10**9
        with binding.Server(sv, pool_bytes=8 << 30) as srv:
            ids = [srv.submit(a, b, m) for a, b, m in zip(lo, hi, mode)]
            mixed = _collect(srv, ids)
            alone = []
            for a, b, m in zip(lo, hi, mode):
                rid = srv.submit(a, b, m)
                alone.append(_collect(srv, [rid])[rid])
        # the regular path, outside the server, for the wide requests
        regular = {}
        for i, (a, b, m) in enumerate(zip(lo, hi, mode)):
            if b - a > ORACLE_MAX_WIDTH:
                regular[i] = (sv.range_count(a, b), sv.range_list(a, b) if m == workloads.MODE_LIST else None)
    base = oracle.base_table(10**9)
    n_oracle = 0
    for i, rid in enumerate(ids):
        (c, lst), (ca, la) = mixed[rid], alone[i]
        assert (c.count, c.checksum) == (ca.count, ca.checksum), i
        if lst is None or la is None:
            assert lst is None and la is None and (mode[i] == workloads.MODE_COUNT or c.count == 0), i
        else:
            np.testing.assert_array_equal(lst, la)
            assert mode[i] == workloads.MODE_LIST and lst.size == c.count
            assert lst.size == 0 or (int(lst[0]) >= lo[i] and int(lst[-1]) < hi[i] and (np.diff(lst) > 0).all())
        if hi[i] - lo[i] <= ORACLE_MAX_WIDTH:
            want = oracle.count_range(lo[i], hi[i], base=base)
            assert (c.count, c.checksum) == want, (i, lo[i], hi[i])
            if mode[i] == workloads.MODE_LIST and want[0]:
                np.testing.assert_array_equal(lst, oracle.list_range(lo[i], hi[i], base=base))
            n_oracle += 1
        else:
            rc, rl = regular[i]
            assert (c.count, c.checksum) == (rc.count, rc.checksum), (i, lo[i], hi[i])
            if rl is not None:
                np.testing.assert_array_equal(lst, rl)
                for x in lst[:: max(1, lst.size // 48)].tolist():
                    assert C.mr_is_prime(int(x)), (i, x)
    assert n_oracle >= 8, n_oracle
