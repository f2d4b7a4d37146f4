"""GPU tests of the autotuners and their cache: the options they pick are
valid and become the context's, and the results computed with them equal the
CPU oracle's (bit-exact: integer results, no tolerance); the JSON cache stores
and restores them per (device, workload)."""
import json

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


def test_autotune_range_result_equals_oracle(torch, tmp_path):
    lo, hi = 10**10 + 3, 10**10 + 2 * 10**9
    with binding.Sieve(10**12) as sv:
        default = sv.options()
        best, ms = sv.autotune_range(lo, hi, reps=1)
        assert ms > 0
        assert sv.options() == best
        assert best["tile_bits"] in (1 << 18, 1 << 19) and best["presieve_groups"] in (5, 6, 7, 8)
        got = sv.range_count(lo, hi)
        assert (got.count, got.checksum) == oracle.count_range(lo, hi)
        a, b = 10**10 + 10**9 - 77, 10**10 + 10**9 + 3_000_000
        np.testing.assert_array_equal(sv.range_list(a, b), oracle.list_range(a, b))
        tot, bins = sv.segment_counts(lo, hi, 1 << 24)
        oc, osum, obins = oracle.segment_counts(lo, hi, 1 << 24)
        assert (tot.count, tot.checksum) == (oc, osum)
        np.testing.assert_array_equal(bins, obins)
        # the cache restores the tuned options into a fresh context
        path = str(tmp_path / "tune.json")
        sv.tune_cache_store(path, "count 1e10+2e9", ms)
        sv.tune_cache_store(path, "other workload", 1.0)
        sv.set_options(cluster_ctas=8, cluster_threshold=16)
        sv.tune_cache_store(path, "cluster segments", 2.0)
    with binding.Sieve(10**12) as sv2:
        assert sv2.options() == default
        assert sv2.tune_cache_load(path, "missing workload") is None
        assert sv2.options() == default
        opts, ms2 = sv2.tune_cache_load(path, "count 1e10+2e9")
        assert opts == best and abs(ms2 - ms) < 1e-3
        doc = json.load(open(path))
        assert len(doc["entries"]) == 3
        got = sv2.range_count(lo, hi)
        assert (got.count, got.checksum) == oracle.count_range(lo, hi)
        opts3, _ = sv2.tune_cache_load(path, "cluster segments")
        assert opts3["cluster_ctas"] == 8 and opts3["cluster_threshold"] == 16
        got = sv2.range_count(lo, hi)
        assert (got.count, got.checksum) == oracle.count_range(lo, hi)
        # a corrupt entry is refused and leaves the options alone
        bad = str(tmp_path / "bad.json")
        with open(path) as f:
            txt = f.read().replace('"tile_bits": ', '"tile_bits": 3')
        with open(bad, "w") as f:
            f.write(txt)
        sv2.set_options(**default)
        with pytest.raises(binding.SieveError):
            sv2.tune_cache_load(bad, "count 1e10+2e9")
        assert sv2.options() == default


def test_autotune_batch_result_equals_oracle(torch):
    q = workloads.batch_queries(n=96, seed=5, lo_exp=(6.0, 12.0), width_exp=(3.0, 6.3))
    with binding.Sieve(int(q.hi.max()) + 1) as sv:
        best, ms = sv.autotune_batch(q.lo, q.hi, q.mode, reps=1)
        assert ms > 0 and sv.options() == best
        cnt, offsets, values = sv.range_batch(q.lo, q.hi, q.mode)
    for i in range(len(q)):
        a, b = int(q.lo[i]), int(q.hi[i])
        want = oracle.count_range(a, b)
        assert (int(cnt[i][0]), int(cnt[i][1])) == want, (i, a, b)
        run = values[int(offsets[i]):int(offsets[i + 1])]
        if q.mode[i] == workloads.MODE_LIST:
            np.testing.assert_array_equal(run, oracle.list_range(a, b))
        else:
            assert run.size == 0
