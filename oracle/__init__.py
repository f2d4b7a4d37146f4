"""CPU oracle for the prime sieve -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this package.  The GPU product path never imports it, and it
never imports the GPU package.

The oracle is the plain definition of Section 1.1 / Figure 1 restricted to a
range [lo, hi) (see oracle.h).  This module is a ctypes wrapper around the C
code; it adds no arithmetic of its own beyond argument marshalling.
"""
from __future__ import annotations

import ctypes
import functools

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID = -1
ERR_RANGE = -2
ERR_CAPACITY = -3
ERR_OOM = -4

_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


class OracleError(RuntimeError):
    pass


class BaseTable:
    """Primes <= limit (Section 1.1), built once and reused across many range calls."""

    def __init__(self, limit: int, oracle: "Oracle | None" = None):
        self.limit = int(limit)
        self.primes = (oracle or default()).primes_upto(self.limit)


class Oracle:
    """ctypes view of one build of oracle.c (the default one, or a test mutant)."""

    def __init__(self, libpath: str):
        lib = ctypes.CDLL(libpath)
        lib.oracle_isqrt.argtypes = [_u64]
        lib.oracle_isqrt.restype = _u64
        lib.oracle_primes_upto.argtypes = [_u64, _p, ctypes.c_size_t]
        lib.oracle_primes_upto.restype = ctypes.c_int64
        lib.oracle_range.argtypes = [_u64, _u64, _p, ctypes.c_size_t, _u64, ctypes.c_int,
                                     _p, _p, _p, ctypes.c_size_t, _p, _u64, _p, ctypes.c_size_t]
        lib.oracle_range.restype = ctypes.c_int
        lib.oracle_is_prime_td.argtypes = [_u64]
        lib.oracle_is_prime_td.restype = ctypes.c_int
        lib.oracle_is_prime_mr.argtypes = [_u64]
        lib.oracle_is_prime_mr.restype = ctypes.c_int
        lib.oracle_first_class_multiple.argtypes = [_u64, _u64, ctypes.c_int, ctypes.c_int]
        lib.oracle_first_class_multiple.restype = _u64
        lib.oracle_default_threads.argtypes = []
        lib.oracle_default_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = libpath

    @staticmethod
    def _check(rc: int, what: str) -> None:
        if rc != OK:
            raise OracleError(f"{what} failed with status {rc}")

    @staticmethod
    def _base_args(base: BaseTable | None):
        if base is None:
            return None, 0, 0
        return base.primes.ctypes.data, base.primes.size, base.limit

    def isqrt(self, n: int) -> int:
        return int(self.lib.oracle_isqrt(n))

    def default_threads(self) -> int:
        return int(self.lib.oracle_default_threads())

    def primes_upto(self, n: int) -> np.ndarray:
        """All primes <= n as uint32 (Section 1.1)."""
        k = self.lib.oracle_primes_upto(n, None, 0)
        if k < 0:
            raise OracleError(f"primes_upto({n}) failed with status {k}")
        out = np.empty(max(k, 1), dtype=np.uint32)
        k2 = self.lib.oracle_primes_upto(n, out.ctypes.data, k)
        if k2 != k:
            raise OracleError(f"primes_upto({n}) failed with status {k2}")
        return out[:k]

    def count_range(self, lo: int, hi: int, base: BaseTable | None = None, threads: int = 0):
        """(count, sum mod 2^64) of the primes in [lo, hi)."""
        c = _u64(0)
        s = _u64(0)
        bp, nb, bl = self._base_args(base)
        rc = self.lib.oracle_range(lo, hi, bp, nb, bl, threads, ctypes.byref(c), ctypes.byref(s),
                                   None, 0, None, 0, None, 0)
        self._check(rc, f"count_range({lo}, {hi})")
        return int(c.value), int(s.value)

    def list_range(self, lo: int, hi: int, base: BaseTable | None = None,
                   threads: int = 0) -> np.ndarray:
        """Primes in [lo, hi), increasing, as uint64."""
        c, _ = self.count_range(lo, hi, base, threads)
        out = np.empty(max(c, 1), dtype=np.uint64)
        n = ctypes.c_size_t(0)
        bp, nb, bl = self._base_args(base)
        rc = self.lib.oracle_range(lo, hi, bp, nb, bl, threads, None, None,
                                   out.ctypes.data, c, ctypes.byref(n), 0, None, 0)
        self._check(rc, f"list_range({lo}, {hi})")
        return out[: n.value]

    def segment_counts(self, lo: int, hi: int, seg_width: int, base: BaseTable | None = None,
                       threads: int = 0):
        """(count, sum, bins): bins[i] counts primes p with p // W - lo // W == i."""
        nb_ = nbins(lo, hi, seg_width)
        bins = np.zeros(max(nb_, 1), dtype=np.uint64)
        c = _u64(0)
        s = _u64(0)
        bp, nb, bl = self._base_args(base)
        rc = self.lib.oracle_range(lo, hi, bp, nb, bl, threads, ctypes.byref(c), ctypes.byref(s),
                                   None, 0, None, seg_width, bins.ctypes.data, nb_)
        self._check(rc, f"segment_counts({lo}, {hi}, {seg_width})")
        return int(c.value), int(s.value), bins[:nb_]

    def is_prime_td(self, n: int) -> bool:
        return bool(self.lib.oracle_is_prime_td(n))

    def is_prime_mr(self, n: int) -> bool:
        return bool(self.lib.oracle_is_prime_mr(n))

    def first_class_multiple(self, M: int, P: int, r: int, from_square: bool = False) -> int:
        return int(self.lib.oracle_first_class_multiple(M, P, r, int(from_square)))

    def raw_range(self, *args) -> int:
        """oracle_range's status code, for argument-error tests."""
        return int(self.lib.oracle_range(*args))


def nbins(lo: int, hi: int, seg_width: int) -> int:
    if hi <= lo:
        return 0
    return (hi - 1) // seg_width - lo // seg_width + 1


@functools.lru_cache(maxsize=1)
def default() -> Oracle:
    return Oracle(_build.build())


@functools.lru_cache(maxsize=4)
def base_table(limit: int) -> BaseTable:
    return BaseTable(limit)


def isqrt(n):
    return default().isqrt(n)


def default_threads():
    return default().default_threads()


def primes_upto(n):
    return default().primes_upto(n)


def count_range(lo, hi, base=None, threads=0):
    return default().count_range(lo, hi, base, threads)


def list_range(lo, hi, base=None, threads=0):
    return default().list_range(lo, hi, base, threads)


def segment_counts(lo, hi, seg_width, base=None, threads=0):
    return default().segment_counts(lo, hi, seg_width, base, threads)


def is_prime_td(n):
    return default().is_prime_td(n)


def is_prime_mr(n):
    return default().is_prime_mr(n)


def first_class_multiple(M, P, r, from_square=False):
    return default().first_class_multiple(M, P, r, from_square)


def raw_range(*args):
    return default().raw_range(*args)


__all__ = [
    "Oracle", "BaseTable", "base_table", "default", "count_range", "list_range",
    "segment_counts", "nbins", "primes_upto", "isqrt", "is_prime_td", "is_prime_mr",
    "first_class_multiple", "default_threads", "OracleError", "raw_range",
]
