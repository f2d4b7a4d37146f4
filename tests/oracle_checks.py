"""Checks that pin the CPU oracle to facts outside itself.

Each check takes an `oracle.Oracle` (the default build, or a deliberately
broken copy made by test_oracle_mutants.py) and raises AssertionError when the
oracle disagrees with:
  * published values (pi(10^n), sums of primes: tests/golden/pi_powers_of_ten.json),
  * the paper's worked example for Table 1 (tests/golden/table1_worked_example.json)
    and the candidate arrays of Figure 2,
  * Python's exact math.isqrt,
  * brute force written here: trial division and a Miller-Rabin test on
    Python integers, both independent of the C code,
  * invariants every answer must have (sorted, 2/3/6k+-1, count == length,
    additivity over adjacent ranges, bins summing to the total).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# independent brute force (Python integers; shares nothing with oracle.c)

def td_is_prime(n: int) -> bool:
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def mr_is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def brute_primes(lo: int, hi: int) -> list[int]:
    """Trial division of every n in [lo, hi) by every d with d*d <= n (numpy, n < 2^62)."""
    if hi <= lo:
        return []
    n = np.arange(lo, hi, dtype=np.int64)
    keep = n >= 2
    d = 2
    while d * d <= hi - 1:
        keep &= (n % d != 0) | (n <= d) | (n < d * d)
        d += 1
    return [int(x) for x in n[keep]]


# ---------------------------------------------------------------------------
# checks

def check_isqrt(o) -> None:
    for n in range(0, 20000):
        assert o.isqrt(n) == math.isqrt(n), n
    rng = np.random.default_rng(7)
    edges = [2**64 - 1, 2**63, 10**18, 10**18 - 1, (2**32 - 1) ** 2, (2**32 - 1) ** 2 - 1]
    for k in rng.integers(1, 2**32 - 1, size=300, dtype=np.uint64):
        k = int(k)
        edges += [k * k - 1, k * k, k * k + 1]
    for n in edges:
        if 0 <= n < 2**64:
            assert o.isqrt(n) == math.isqrt(n), n


def check_primes_upto_small(o) -> None:
    for n in list(range(0, 200)) + [961, 962, 1023, 1024, 4096, 9973, 10000]:
        got = o.primes_upto(n).tolist()
        assert got == brute_primes(2, n + 1), n


def check_primes_upto_published(o) -> None:
    g = golden("pi_powers_of_ten.json")
    for e in range(1, 9):
        p = o.primes_upto(10**e)
        assert p.size == g["pi"][str(e)], e
        assert int(p.astype(np.uint64).sum()) == g["sum_below"][str(e)], e


def check_range_small_bruteforce(o) -> None:
    rng = np.random.default_rng(11)
    cases = [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (2, 3), (3, 4), (1, 2), (4, 5), (5, 6),
             (0, 26), (0, 25), (24, 26), (25, 26), (26, 50), (48, 50), (120, 122),
             (0, 170), (168, 170), (5, 1000), (10**6 - 100, 10**6 + 100)]
    # ranges that end exactly after, or start exactly at, a prime square p^2
    for p in (2, 3, 5, 7, 11, 13, 31, 97, 997):
        cases += [(p * p - 3, p * p + 1), (p * p, p * p + 2), (p * p - 1, p * p), (p, p * p + 1)]
    for _ in range(60):
        lo = int(rng.integers(0, 10**6))
        cases.append((lo, lo + int(rng.integers(0, 3000))))
    for lo, hi in cases:
        want = brute_primes(lo, hi)
        for threads in (1, 3):
            c, s = o.count_range(lo, hi, threads=threads)
            assert c == len(want), (lo, hi, threads)
            assert s == sum(want) % 2**64, (lo, hi, threads)
            got = o.list_range(lo, hi, threads=threads).tolist()
            assert got == want, (lo, hi, threads)


def check_range_published(o) -> None:
    g = golden("pi_powers_of_ten.json")
    for e in range(1, 10):
        c, s = o.count_range(2, 10**e + 1)
        assert c == g["pi"][str(e)], e
        assert s == g["sum_below"][str(e)], e


def check_range_1e10(o) -> None:
    g = golden("pi_powers_of_ten.json")
    c, s = o.count_range(2, 10**10 + 1)
    assert c == g["pi"]["10"]
    assert s == g["sum_below"]["10"]


def check_high_windows_mr(o) -> None:
    """Windows near 1e12 and 1e15: every integer classified by Miller-Rabin."""
    for lo, width in ((10**12 - 1000, 2000), (10**15 - 700, 1500), (2**40 + 12345, 1500)):
        hi = lo + width
        from oracle import BaseTable  # local import keeps this module dependency-free
        base = BaseTable(math.isqrt(hi - 1), o)
        got = o.list_range(lo, hi, base=base).tolist()
        want = [n for n in range(lo, hi) if mr_is_prime(n)]
        assert got == want, lo
        c, s = o.count_range(lo, hi, base=base)
        assert c == len(want) and s == sum(want) % 2**64, lo


def check_invariants(o) -> None:
    lst = o.list_range(0, 2_000_000).astype(np.int64)
    assert lst[0] == 2 and lst[1] == 3
    assert np.all(np.diff(lst) > 0)
    r = lst[2:] % 6
    assert np.all((r == 1) | (r == 5))
    c, s = o.count_range(0, 2_000_000)
    assert c == lst.size and s == int(lst.sum()) % 2**64
    # additivity over adjacent ranges
    for a, b, cc in ((2, 777_777, 1_999_999), (10**9, 10**9 + 12_345, 10**9 + 3_000_000)):
        c1, s1 = o.count_range(a, b)
        c2, s2 = o.count_range(b, cc)
        c3, s3 = o.count_range(a, cc)
        assert c1 + c2 == c3 and (s1 + s2) % 2**64 == s3


def check_segment_bins(o) -> None:
    for lo, hi, w in ((2, 10**7 + 1, 1 << 20), (12_345, 5_000_000, 999_983), (0, 100, 7),
                      (10**9 - 5, 10**9 + 2_000_000, 1 << 18)):
        c, s, bins = o.segment_counts(lo, hi, w)
        assert int(bins.sum()) == c
        cc, ss = o.count_range(lo, hi)
        assert (c, s) == (cc, ss)
        first = lo // w
        for i in range(len(bins)):
            a = max(lo, (first + i) * w)
            b = min(hi, (first + i + 1) * w)
            assert int(bins[i]) == o.count_range(a, b)[0], (lo, hi, w, i)


def check_mr_vs_td(o) -> None:
    for n in range(0, 30000):
        assert o.is_prime_mr(n) == td_is_prime(n), n
        assert o.is_prime_td(n) == td_is_prime(n), n
    # strong pseudoprimes to several small bases, Carmichael numbers, big primes
    composites = [561, 1105, 1729, 2047, 3215031751, 3825123056546413051,
                  2**61 + 1, (2**31 - 1) * (2**31 + 11)]
    for n in composites:
        assert o.is_prime_mr(n) == mr_is_prime(n), n
    primes = [2**61 - 1, 2**31 - 1, 10**18 + 3, 18446744073709551557]
    for n in primes:
        assert o.is_prime_mr(n) and mr_is_prime(n), n
    rng = np.random.default_rng(3)
    for n in rng.integers(2**40, 2**63, size=400, dtype=np.uint64):
        assert o.is_prime_mr(int(n)) == mr_is_prime(int(n)), int(n)


def check_first_class_multiple(o) -> None:
    ex = golden("table1_worked_example.json")
    assert o.first_class_multiple(ex["M"], ex["P"], 1) == ex["start_value_1"]
    assert o.first_class_multiple(ex["M"], ex["P"], 5) == ex["start_value_5"]
    rng = np.random.default_rng(5)
    primes = [p for p in range(5, 400) if td_is_prime(p)]
    for P in primes:
        for M in [int(x) for x in rng.integers(0, 10**6, size=5)] + [0, 1, P, P * P, P * P + 1]:
            for r in (1, 5):
                for sq in (False, True):
                    start = max(M, P * P) if sq else M
                    v = start
                    while not (v % P == 0 and v % 6 == r):
                        v += 1
                    assert o.first_class_multiple(M, P, r, sq) == v, (M, P, r, sq)
    # Section 2.4: sieving starts at P^2; for class 5 that is P^2 + 4P or P^2 + 2P
    assert o.first_class_multiple(0, 5, 5, True) == 35
    assert o.first_class_multiple(0, 7, 5, True) == 77
    assert o.first_class_multiple(0, 7, 1, True) == 49


def check_figure2(o) -> None:
    f2 = golden("figure2_residue_arrays.json")
    survivors_one = [v for v in f2["A_one"] if v in set(o.list_range(0, 50).tolist())]
    assert survivors_one == [7, 13, 19, 31, 37, 43]      # 25 = 5*5 is struck
    survivors_five = [v for v in f2["A_five"] if v in set(o.list_range(0, 50).tolist())]
    assert survivors_five == [5, 11, 17, 23, 29, 41]     # 35 = 5*7 is struck
    assert all(v % 6 == 1 for v in f2["A_one"]) and all(v % 6 == 5 for v in f2["A_five"])


def check_argument_errors(o) -> None:
    import oracle as _o
    assert o.raw_range(5, 4, None, 0, 0, 1, None, None, None, 0, None, 0, None, 0) == _o.ERR_INVALID
    base = o.primes_upto(100)
    # a base table that stops short of isqrt(hi - 1) is refused
    assert o.raw_range(0, 10**6, base.ctypes.data, base.size, 100, 1,
                       None, None, None, 0, None, 0, None, 0) == _o.ERR_RANGE
    # capacity: a list that does not fit is refused and reports the needed size
    import ctypes
    out = np.zeros(3, dtype=np.uint64)
    n = ctypes.c_size_t(0)
    assert o.raw_range(0, 100, None, 0, 0, 1, None, None, out.ctypes.data, 3, ctypes.byref(n),
                       0, None, 0) == _o.ERR_CAPACITY
    assert n.value == 25


ALL_FAST_CHECKS = [check_isqrt, check_primes_upto_small, check_primes_upto_published, check_range_small_bruteforce,
                   check_range_published, check_high_windows_mr, check_invariants,
                   check_segment_bins, check_mr_vs_td, check_first_class_multiple, check_figure2,
                   check_argument_errors]
