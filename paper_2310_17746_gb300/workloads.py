"""Seeded synthetic workloads shared by the GPU path's tests/benchmarks and the oracle.

This module holds no sieve arithmetic: it only draws query ranges, modes and
arrival times from numpy's PCG64 generator, so that both sides see the same
inputs.  The paper measures no public dataset; its experiments sieve [2, N]
for growing N (Section 5), so the range workloads below are plain intervals and
the query workloads are synthetic mixes of narrow and wide ranges at high
offsets.

Recipes:
  * plain range      [2, 1e8]            list mode, uint32 output
  * segmented count  [2, 1e10]           count + per-2^24-number segment counts
  * headline count   [2, 1e12]           count + per-2^30-number block histogram
  * batch            4096 queries, seed 0: lo = floor(10^U(6, 15)),
                     width = floor(10^U(3, 8)), hi = lo + width; exactly half
                     count mode and half list mode, in shuffled order
  * serving          seed 1: lo = floor(10^U(6, 18)), width = floor(10^U(3, 9)),
                     list mode with probability 0.2, exponential inter-arrival
                     gaps at rate lam requests/s
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MODE_COUNT = 0
MODE_LIST = 1


@dataclass(frozen=True)
class RangeWorkload:
    name: str
    lo: int
    hi: int          # exclusive
    seg_width: int   # 0: no per-segment counts
    mode: int


PLAIN_1E8 = RangeWorkload("plain sieve [2, 1e8] (uint32 list)", 2, 10**8 + 1, 0, MODE_LIST)
SEGMENTED_1E10 = RangeWorkload("segmented count [2, 1e10], 2^24-number segments",
                               2, 10**10 + 1, 1 << 24, MODE_COUNT)
COUNT_1E12 = RangeWorkload("count [2, 1e12], 2^30-number block histogram",
                           2, 10**12 + 1, 1 << 30, MODE_COUNT)


@dataclass
class QuerySet:
    lo: np.ndarray    # uint64
    hi: np.ndarray    # uint64, exclusive
    mode: np.ndarray  # uint8, MODE_COUNT / MODE_LIST

    def __len__(self) -> int:
        return int(self.lo.size)

    def subset(self, idx) -> "QuerySet":
        return QuerySet(self.lo[idx].copy(), self.hi[idx].copy(), self.mode[idx].copy())


def _log_uniform_int(rng: np.random.Generator, n: int, e_lo: float, e_hi: float) -> np.ndarray:
    x = rng.uniform(e_lo, e_hi, size=n)
    return np.floor(np.power(10.0, x)).astype(np.uint64)


def batch_queries(n: int = 4096, seed: int = 0, lo_exp=(6.0, 15.0), width_exp=(3.0, 8.0),
                  list_fraction: float = 0.5) -> QuerySet:
    """Batched-range workload: log-uniform lo and width, exact list/count split."""
    rng = np.random.default_rng(seed)
    lo = _log_uniform_int(rng, n, *lo_exp)
    width = _log_uniform_int(rng, n, *width_exp)
    n_list = int(round(n * list_fraction))
    mode = np.zeros(n, dtype=np.uint8)
    mode[n - n_list:] = MODE_LIST
    rng.shuffle(mode)
    return QuerySet(lo, lo + width, mode)


@dataclass
class Arrivals:
    queries: QuerySet
    t_arrive: np.ndarray  # float64 seconds from the start, increasing
    rate: float


def serving_arrivals(rate: float, n: int, seed: int = 1, lo_exp=(6.0, 18.0),
                     width_exp=(3.0, 9.0), list_prob: float = 0.2) -> Arrivals:
    """Open-loop Poisson request stream at `rate` requests/s."""
    rng = np.random.default_rng(seed)
    lo = _log_uniform_int(rng, n, *lo_exp)
    width = _log_uniform_int(rng, n, *width_exp)
    mode = (rng.uniform(0.0, 1.0, size=n) < list_prob).astype(np.uint8)
    gaps = rng.exponential(1.0 / rate, size=n)
    return Arrivals(QuerySet(lo, lo + width, mode), np.cumsum(gaps), float(rate))


def random_small_ranges(n: int, seed: int, max_lo: int, max_width: int) -> QuerySet:
    """Uniform small ranges for edge/parity sweeps (lo in [0, max_lo], width in [0, max_width])."""
    rng = np.random.default_rng(seed)
    lo = rng.integers(0, max_lo + 1, size=n, dtype=np.uint64)
    width = rng.integers(0, max_width + 1, size=n, dtype=np.uint64)
    mode = rng.integers(0, 2, size=n, dtype=np.uint8)
    return QuerySet(lo, lo + width, mode)
