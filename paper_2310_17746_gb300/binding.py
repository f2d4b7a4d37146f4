"""ctypes binding of libsieve_gb300.so (include/sieve.h), argument marshalling only.

Every step of the sieve runs in the library's CUDA kernels; this module only
converts Python ints, numpy arrays (host buffers) and torch CUDA tensors
(device buffers) into the C ABI's pointers and sizes.  There is no CPU
fallback: if the library cannot be built or loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import functools
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK = 0
PENDING = 1
ERR_INVALID = -1
ERR_RANGE = -2
ERR_CAPACITY = -3
ERR_OOM = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_BUSY = -7
ERR_NOT_FOUND = -8

COUNT = 0
LIST = 1
OUT_DEVICE = 1
ASYNC = 2

_STATUS_NAMES = {OK: "OK", PENDING: "PENDING", ERR_INVALID: "INVALID", ERR_RANGE: "RANGE",
                 ERR_CAPACITY: "CAPACITY", ERR_OOM: "OOM", ERR_CUDA: "CUDA",
                 ERR_TIMEOUT: "TIMEOUT", ERR_BUSY: "BUSY", ERR_NOT_FOUND: "NOT_FOUND"}


class SieveError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {message}")


class CountResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("checksum", ctypes.c_uint64)]


class Options(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("group_hits", ctypes.c_uint32),
                ("presieve_groups", ctypes.c_uint32), ("batch_tile_bits", ctypes.c_uint32),
                ("chunk_primes", ctypes.c_uint32), ("bucket_threshold", ctypes.c_uint32),
                ("bucket_wave", ctypes.c_uint32), ("bucket_scatter", ctypes.c_uint32),
                ("list_single_pass", ctypes.c_uint32), ("cluster_ctas", ctypes.c_uint32),
                ("cluster_threshold", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"tile_bits": self.tile_bits, "block_threads": self.block_threads,
                "ctas_per_sm": self.ctas_per_sm, "group_hits": self.group_hits,
                "presieve_groups": self.presieve_groups, "batch_tile_bits": self.batch_tile_bits,
                "chunk_primes": self.chunk_primes, "bucket_threshold": self.bucket_threshold,
                "bucket_wave": self.bucket_wave, "bucket_scatter": self.bucket_scatter,
                "list_single_pass": self.list_single_pass, "cluster_ctas": self.cluster_ctas,
                "cluster_threshold": self.cluster_threshold}


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_size_t),
                ("max_queue", ctypes.c_size_t), ("batch_scratch_bytes", ctypes.c_size_t)]


class PhaseTimes(ctypes.Structure):
    _fields_ = [("sieve_ms", ctypes.c_double), ("scan_ms", ctypes.c_double), ("compact_ms", ctypes.c_double),
                ("tiles", ctypes.c_uint64), ("tile_len", ctypes.c_uint64), ("listed", ctypes.c_uint64),
                ("bucket_waves", ctypes.c_uint64), ("cluster_ctas", ctypes.c_uint64),
                ("batch_plan_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("overlapped_batches", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("pool_used_bytes", ctypes.c_uint64), ("mean_batch", ctypes.c_double),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_p = ctypes.c_void_p
_i = ctypes.c_int
_u = ctypes.c_uint

# name -> (restype, argtypes); every entry is declared in include/sieve.h
SIGNATURES = {
    "sieve_create": (_i, [ctypes.POINTER(_p), _u64, _i, _p]),
    "sieve_destroy": (None, [_p]),
    "sieve_set_stream": (_i, [_p, _p]),
    "sieve_get_options": (_i, [_p, ctypes.POINTER(Options)]),
    "sieve_set_options": (_i, [_p, ctypes.POINTER(Options)]),
    "sieve_base_table": (_i, [_p, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_p)]),
    "sieve_launch_count": (_u64, [_p]),
    "sieve_last_error": (ctypes.c_char_p, []),
    "sieve_count": (_i, [_p, _u64, ctypes.POINTER(CountResult)]),
    "sieve_primes": (_i, [_p, _u64, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_primes_u32": (_i, [_p, _u64, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_range": (_i, [_p, _u64, _u64, _i, _p, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_segment_counts": (_i, [_p, _u64, _u64, _u64, _p, _sz, _p, _u]),
    "sieve_table1_start": (_i, [_u64, _u64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64)]),
    "sieve_inverse6_start": (_i, [_u64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_uint32)]),
    "sieve_range_list_noalloc": (_i, [_p, _u64, _u64, _p, _sz, ctypes.POINTER(_sz), _p]),
    "sieve_range_batch": (_i, [_p, _p, _p, _p, _sz, _p, _p, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_range_each": (_i, [_p, _p, _p, _p, _sz, _p, _p, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_autotune_batch": (_i, [_p, _p, _p, _p, _sz, _i, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_double)]),
    "sieve_autotune_range": (_i, [_p, _u64, _u64, _i, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_double)]),
    "sieve_server_start": (_i, [_p, ctypes.POINTER(ServerConfig), ctypes.POINTER(_p)]),
    "sieve_server_submit": (_i, [_p, _u64, _u64, _i, ctypes.POINTER(_u64)]),
    "sieve_server_poll": (_i, [_p, _u64, _p, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_server_next_done": (_i, [_p, ctypes.POINTER(_u64), _i]),
    "sieve_server_get_stats": (_i, [_p, ctypes.POINTER(ServerStats), _i]),
    "sieve_server_stop": (None, [_p]),
    "sieve_measure_smem_atomics": (_i, [_i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "sieve_set_phase_timing": (_i, [_p, _i]),
    "sieve_get_phase_times": (_i, [_p, _p]),
    "sieve_next": (_i, [_p, _u64, _sz, _p, ctypes.POINTER(_sz), _u]),
    "sieve_count_checkpointed": (_i, [_p, _u64, _u64, _u64, _u64, ctypes.c_char_p, _p, _sz, _p, _u64,
                                      ctypes.POINTER(_u64)]),
    "sieve_primes_to_file": (_i, [_p, _u64, _u64, ctypes.c_char_p, _sz, _i, _u64, ctypes.POINTER(_u64)]),
    "sieve_range_naive": (_i, [_p, _u64, _u64, _i, _p, _p, _sz, ctypes.POINTER(_sz), _u]),
    "sieve_tune_cache_store": (_i, [_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_double]),
    "sieve_tune_cache_load": (_i, [_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(_i),
                                   ctypes.POINTER(ctypes.c_double)]),
}


@functools.lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    """Build (if the sources changed) and load the CUDA library."""
    path = _build.build()
    handle = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(handle, name)
        fn.restype = res
        fn.argtypes = args
    return handle


def last_error() -> str:
    msg = lib().sieve_last_error()
    return msg.decode() if msg else ""


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise SieveError(rc, where, last_error())
    return rc


def table1_start(B: int, M: int, P: int) -> tuple[int, int]:
    """Host evaluation of the kernels' Table 1 start-index routine."""
    a = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(lib().sieve_table1_start(B, M, P, ctypes.byref(a), ctypes.byref(b)), "sieve_table1_start")
    return a.value, b.value


def inverse6_start(B: int, P: int) -> tuple[int, int]:
    """Host evaluation of the kernels' inverse-of-6 start-index routine."""
    a = ctypes.c_uint32(0)
    b = ctypes.c_uint32(0)
    _check(lib().sieve_inverse6_start(B, P, ctypes.byref(a), ctypes.byref(b)), "sieve_inverse6_start")
    return a.value, b.value


def measure_smem_atomics(device: int = 0) -> tuple[float, float]:
    """(conflict-free, random-bank) shared-memory atomic AND throughput of the
    device, in lane operations per SM per clock."""
    a = ctypes.c_double(0.0)
    b = ctypes.c_double(0.0)
    _check(lib().sieve_measure_smem_atomics(int(device), ctypes.byref(a), ctypes.byref(b)),
           "sieve_measure_smem_atomics")
    return a.value, b.value


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


_TORCH_INT_DTYPES = {"torch.int64": 8, "torch.uint64": 8, "torch.int32": 4, "torch.uint32": 4}


def _ptr_and_flag(x, esizes=(8,), min_numel: int = 0, what: str = "buffer"):
    """(pointer, flags, capacity in elements) for an output buffer: a torch
    CUDA tensor or a numpy array of integers whose element size is one of
    `esizes` bytes, contiguous, with at least `min_numel` elements.  Anything
    else raises before the library is called, so that a kernel never writes
    past a buffer that is smaller than its element count suggests."""
    if x is None:
        return None, 0, 0
    if _is_torch_cuda(x):
        esize = _TORCH_INT_DTYPES.get(str(x.dtype))
        if esize is None or esize not in esizes or x.element_size() != esize:
            raise TypeError(f"{what}: device buffer must be an integer tensor of {' or '.join(map(str, esizes))}"
                            f"-byte elements, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{what}: device buffers must be contiguous")
        n = int(x.numel())
        if n < min_numel:
            raise ValueError(f"{what}: device buffer needs at least {min_numel} elements, has {n}")
        return x.data_ptr(), OUT_DEVICE, n
    if isinstance(x, np.ndarray):
        if x.dtype.kind not in "iu" or x.dtype.itemsize not in esizes:
            raise TypeError(f"{what}: host buffer must be an integer array of "
                            f"{' or '.join(map(str, esizes))}-byte elements, got {x.dtype}")
        if not x.flags.c_contiguous or not x.flags.writeable:
            raise ValueError(f"{what}: host buffers must be C-contiguous and writeable")
        if x.size < min_numel:
            raise ValueError(f"{what}: host buffer needs at least {min_numel} elements, has {x.size}")
        return x.ctypes.data, 0, int(x.size)
    raise TypeError(f"{what}: expected a numpy array or a torch CUDA tensor")


def _current_stream_handle(device: int):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except ImportError:
        pass
    return None


@dataclass
class CountAndSum:
    count: int
    checksum: int


class Sieve:
    """One library context: base table of primes <= isqrt(max_hi - 1) on `device`."""

    def __init__(self, max_hi: int, device: int = 0, stream=None):
        if stream is None:
            stream = _current_stream_handle(device)
        self._lib = lib()
        h = _p()
        _check(self._lib.sieve_create(ctypes.byref(h), int(max_hi), int(device), stream), "sieve_create")
        self._h = h
        self.device = device
        self.max_hi = int(max_hi)

    # lifetime -------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.sieve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # configuration ----------------------------------------------------------
    def set_stream(self, stream_handle) -> None:
        _check(self._lib.sieve_set_stream(self._h, stream_handle), "sieve_set_stream")

    def options(self) -> dict:
        o = Options()
        _check(self._lib.sieve_get_options(self._h, ctypes.byref(o)), "sieve_get_options")
        return o.as_dict()

    def set_options(self, **kw) -> None:
        o = Options()
        _check(self._lib.sieve_get_options(self._h, ctypes.byref(o)), "sieve_get_options")
        for k, v in kw.items():
            setattr(o, k, int(v))
        _check(self._lib.sieve_set_options(self._h, ctypes.byref(o)), "sieve_set_options")

    def set_phase_timing(self, enable: bool = True) -> None:
        """Turn per-phase timing of single-range and batch calls on or off."""
        _check(self._lib.sieve_set_phase_timing(self._h, 1 if enable else 0), "sieve_set_phase_timing")

    def phase_times(self) -> dict:
        """Device times (ms) of the last single-range call's tile kernel, scan
        and compaction, with its tile count, tile length and listed primes;
        after a batch call, its graph's device time (sieve_ms) and its host
        planning time (batch_plan_ms)."""
        t = PhaseTimes()
        _check(self._lib.sieve_get_phase_times(self._h, ctypes.byref(t)), "sieve_get_phase_times")
        return {k: getattr(t, k) for k, _ in PhaseTimes._fields_}

    def base_table(self) -> tuple[int, int, int]:
        lim = _u64(0)
        n = _u64(0)
        ptr = _p()
        _check(self._lib.sieve_base_table(self._h, ctypes.byref(lim), ctypes.byref(n), ctypes.byref(ptr)),
               "sieve_base_table")
        return lim.value, n.value, ptr.value or 0

    def launch_count(self) -> int:
        return int(self._lib.sieve_launch_count(self._h))

    # calls ------------------------------------------------------------------
    def count(self, n: int) -> CountAndSum:
        r = CountResult()
        _check(self._lib.sieve_count(self._h, int(n), ctypes.byref(r)), "sieve_count")
        return CountAndSum(r.count, r.checksum)

    def primes(self, n: int, out=None, dtype=np.uint64):
        """Primes <= n.  With `out` (numpy array or torch CUDA tensor of 4- or
        8-byte integers) the list goes there and the count is returned;
        without it a new numpy array is returned."""
        if out is None:
            c = self.count(n).count
            out = np.empty(max(c, 1), dtype=dtype)
            got = self.primes(n, out)
            return out[:got]
        ptr, flags, cap = _ptr_and_flag(out, (4, 8), what="out")
        nout = _sz(0)
        esize = out.element_size() if _is_torch_cuda(out) else out.itemsize
        fn = self._lib.sieve_primes_u32 if esize == 4 else self._lib.sieve_primes
        _check(fn(self._h, int(n), ptr, cap, ctypes.byref(nout), flags), "sieve_primes")
        return int(nout.value)

    def range_count(self, lo: int, hi: int, out=None, asynchronous: bool = False):
        """(count, checksum) of primes in [lo, hi).  With `out` = a torch CUDA
        int64 tensor of 2 elements the result is written there (and the call
        is only enqueued when asynchronous=True)."""
        if out is not None:
            if not _is_torch_cuda(out):
                raise TypeError("out: expected a torch CUDA int64 tensor of 2 elements")
            ptr, flags, _ = _ptr_and_flag(out, (8,), 2, what="out")
            if asynchronous:
                flags |= ASYNC
            _check(self._lib.sieve_range(self._h, int(lo), int(hi), COUNT, ptr, None, 0, None, flags),
                   "sieve_range")
            return None
        r = CountResult()
        _check(self._lib.sieve_range(self._h, int(lo), int(hi), COUNT, ctypes.cast(ctypes.byref(r), _p),
                                     None, 0, None, 0), "sieve_range")
        return CountAndSum(r.count, r.checksum)

    def range_list(self, lo: int, hi: int, out=None):
        """Primes in [lo, hi) as uint64: into `out` (returns the count) or a new array."""
        if out is None:
            c = self.range_count(lo, hi).count
            out = np.empty(max(c, 1), dtype=np.uint64)
            got = self.range_list(lo, hi, out)
            return out[:got]
        ptr, flags, cap = _ptr_and_flag(out, (8,), what="out")
        nout = _sz(0)
        _check(self._lib.sieve_range(self._h, int(lo), int(hi), LIST, None, ptr, cap, ctypes.byref(nout), flags),
               "sieve_range")
        return int(nout.value)

    def naive_count(self, lo: int, hi: int) -> CountAndSum:
        """(count, checksum) of [lo, hi) by the plain global-bitmap GPU sieve
        (sieve_range_naive), the comparison point for the segmented path."""
        r = CountResult()
        _check(self._lib.sieve_range_naive(self._h, int(lo), int(hi), COUNT, ctypes.cast(ctypes.byref(r), _p),
                                           None, 0, None, 0), "sieve_range_naive")
        return CountAndSum(r.count, r.checksum)

    def naive_list(self, lo: int, hi: int, out=None):
        """Primes in [lo, hi) as uint64 by the plain GPU sieve: into `out`
        (numpy uint64 or torch CUDA int64; returns the count) or a new array."""
        if out is None:
            c = self.naive_count(lo, hi).count
            out = np.empty(max(c, 1), dtype=np.uint64)
            got = self.naive_list(lo, hi, out)
            return out[:got]
        ptr, flags, cap = _ptr_and_flag(out, (8,), what="out")
        nout = _sz(0)
        _check(self._lib.sieve_range_naive(self._h, int(lo), int(hi), LIST, None, ptr, cap, ctypes.byref(nout),
                                           flags), "sieve_range_naive")
        return int(nout.value)

    def next_primes(self, after: int, k: int, out=None):
        """The first k primes greater than `after` (incremental: the base
        table grows as needed).  Into `out` (numpy uint64 or torch CUDA int64;
        returns the number written) or a new numpy array."""
        if out is None:
            out = np.empty(max(int(k), 1), dtype=np.uint64)
            n = self.next_primes(after, k, out)
            return out[:n]
        ptr, flags, cap = _ptr_and_flag(out, (8,), what="out")
        if k > cap:
            raise ValueError("out holds fewer than k elements")
        nout = _sz(0)
        _check(self._lib.sieve_next(self._h, int(after), int(k), ptr, ctypes.byref(nout), flags), "sieve_next")
        return int(nout.value)

    def range_list_noalloc(self, lo: int, hi: int, out) -> tuple[int, CountAndSum]:
        """Primes in [lo, hi) into the torch CUDA int64 tensor `out` through the
        entry point that allocates nothing; returns (number, count/checksum)."""
        if not _is_torch_cuda(out):
            raise TypeError("out must be a torch CUDA tensor")
        ptr, _, cap = _ptr_and_flag(out, (8,), what="out")
        nout = _sz(0)
        r = CountResult()
        _check(self._lib.sieve_range_list_noalloc(self._h, int(lo), int(hi), ptr, cap,
                                                  ctypes.byref(nout), ctypes.cast(ctypes.byref(r), _p)),
               "sieve_range_list_noalloc")
        return int(nout.value), CountAndSum(r.count, r.checksum)

    def _batch_call(self, fname, lo, hi, mode, cnt, offsets, values):
        lo = np.ascontiguousarray(lo, dtype=np.uint64)
        hi = np.ascontiguousarray(hi, dtype=np.uint64)
        mode = np.ascontiguousarray(mode, dtype=np.uint8)
        nq = lo.size
        if hi.size != nq or mode.size != nq:
            raise ValueError("lo, hi and mode must have the same length")
        flags = 0
        if _is_torch_cuda(cnt) or _is_torch_cuda(offsets) or _is_torch_cuda(values):
            if not (_is_torch_cuda(cnt) and _is_torch_cuda(offsets) and (values is None or _is_torch_cuda(values))):
                raise TypeError("device mode needs cnt, offsets (and values) as torch CUDA tensors")
            flags = OUT_DEVICE
        vptr, _, cap = _ptr_and_flag(values, (8,), what="values")
        cptr = _ptr_and_flag(cnt, (8,), 2 * nq, what="cnt")[0]
        optr = _ptr_and_flag(offsets, (8,), nq + 1, what="offsets")[0]
        nout = _sz(0)
        rc = getattr(self._lib, fname)(self._h, lo.ctypes.data, hi.ctypes.data, mode.ctypes.data, nq,
                                       cptr, optr, vptr, cap, ctypes.byref(nout), flags)
        return rc, int(nout.value)

    def range_batch(self, lo, hi, mode, cnt=None, offsets=None, values=None, naive: bool = False):
        """Many queries [lo[i], hi[i]) in one batched launch (mode[i]: COUNT or LIST).

        Host mode (cnt/offsets/values None or numpy): returns (cnt, offsets,
        values) as numpy uint64 arrays -- cnt[i] = (count, checksum), query
        i's primes (list mode) at values[offsets[i]:offsets[i+1]].  Device
        mode (torch CUDA tensors: cnt int64 (nq, 2), offsets int64 (nq + 1),
        values int64): fills them and returns the number of listed primes.
        naive=True answers with one range launch per query instead."""
        fname = "sieve_range_each" if naive else "sieve_range_batch"
        nq = int(np.asarray(lo).size)
        if _is_torch_cuda(cnt):
            rc, n = self._batch_call(fname, lo, hi, mode, cnt, offsets, values)
            _check(rc, fname)
            return n
        cnt = np.zeros((nq, 2), dtype=np.uint64) if cnt is None else cnt
        offsets = np.zeros(nq + 1, dtype=np.uint64) if offsets is None else offsets
        if values is None:
            rc, n = self._batch_call(fname, lo, hi, mode, cnt, offsets, None)
            if rc == ERR_CAPACITY:
                values = np.empty(max(n, 1), dtype=np.uint64)
                rc, n = self._batch_call(fname, lo, hi, mode, cnt, offsets, values)
            else:
                values = np.empty(0, dtype=np.uint64)
        else:
            rc, n = self._batch_call(fname, lo, hi, mode, cnt, offsets, values)
        _check(rc, fname)
        return cnt, offsets, values[:n]

    def autotune_batch(self, lo, hi, mode, reps: int = 2) -> tuple[dict, float]:
        """Time the batch call over its tunables on these queries; the fastest
        setting becomes the context's.  Returns (options, milliseconds)."""
        lo = np.ascontiguousarray(lo, dtype=np.uint64)
        hi = np.ascontiguousarray(hi, dtype=np.uint64)
        mode = np.ascontiguousarray(mode, dtype=np.uint8)
        o = Options()
        ms = ctypes.c_double(0.0)
        _check(self._lib.sieve_autotune_batch(self._h, lo.ctypes.data, hi.ctypes.data, mode.ctypes.data, lo.size,
                                              int(reps), ctypes.byref(o), ctypes.byref(ms)), "sieve_autotune_batch")
        return o.as_dict(), float(ms.value)

    def autotune_range(self, lo: int, hi: int, reps: int = 2) -> tuple[dict, float]:
        """Time the count kernel over its tunables on [lo, hi); the fastest
        setting becomes the context's.  Returns (options, milliseconds)."""
        o = Options()
        ms = ctypes.c_double(0.0)
        _check(self._lib.sieve_autotune_range(self._h, int(lo), int(hi), int(reps), ctypes.byref(o),
                                              ctypes.byref(ms)), "sieve_autotune_range")
        return o.as_dict(), float(ms.value)

    def count_checkpointed(self, lo: int, hi: int, seg_width: int, chunk_width: int, state_path: str,
                           max_chunks: int = 0):
        """Checkpointed count of [lo, hi) (sieve_count_checkpointed).  Returns
        (done, CountAndSum, bins, next): done is False when max_chunks stopped
        the call early (the state file holds the progress)."""
        nb = self.nbins(lo, hi, seg_width) if seg_width else 0
        bins = np.zeros(max(nb, 1), dtype=np.uint64)
        r = CountResult()
        nxt = _u64(0)
        rc = self._lib.sieve_count_checkpointed(self._h, int(lo), int(hi), int(seg_width), int(chunk_width),
                                                str(state_path).encode(), bins.ctypes.data, nb,
                                                ctypes.cast(ctypes.byref(r), _p), int(max_chunks), ctypes.byref(nxt))
        _check(rc, "sieve_count_checkpointed")
        return rc == OK, CountAndSum(r.count, r.checksum), bins[:nb], int(nxt.value)

    def primes_to_file(self, lo: int, hi: int, path: str, segment_primes: int = 0, resume: bool = False,
                       max_segments: int = 0):
        """Primes of [lo, hi) spilled to the uint64 file `path` in store
        segments (sieve_primes_to_file).  Returns (done, primes written)."""
        n = _u64(0)
        rc = self._lib.sieve_primes_to_file(self._h, int(lo), int(hi), str(path).encode(), int(segment_primes),
                                            1 if resume else 0, int(max_segments), ctypes.byref(n))
        _check(rc, "sieve_primes_to_file")
        return rc == OK, int(n.value)

    def tune_cache_store(self, path: str, workload: str, ms: float = 0.0) -> None:
        """Save the context's current options in the JSON tuning cache at
        `path` under (this device, its SM count, `workload`)."""
        _check(self._lib.sieve_tune_cache_store(self._h, str(path).encode(), workload.encode(), float(ms)),
               "sieve_tune_cache_store")

    def tune_cache_load(self, path: str, workload: str):
        """Options from the tuning cache for (this device, `workload`): made
        the context's and returned as (options, ms); None if absent."""
        found = _i(0)
        ms = ctypes.c_double(0.0)
        _check(self._lib.sieve_tune_cache_load(self._h, str(path).encode(), workload.encode(), ctypes.byref(found),
                                               ctypes.byref(ms)), "sieve_tune_cache_load")
        return (self.options(), float(ms.value)) if found.value else None

    @staticmethod
    def nbins(lo: int, hi: int, seg_width: int) -> int:
        return 0 if hi <= lo else (hi - 1) // seg_width - lo // seg_width + 1

    def segment_counts(self, lo: int, hi: int, seg_width: int, counts=None, total=None,
                       asynchronous: bool = False):
        """Per-segment counts of the primes in [lo, hi).  Host mode (counts None
        or numpy): returns (CountAndSum, counts).  Device mode (counts and total
        torch CUDA int64 tensors): fills them and returns None."""
        nb = self.nbins(lo, hi, seg_width)
        if counts is not None and _is_torch_cuda(counts):
            cptr, flags, _ = _ptr_and_flag(counts, (8,), nb, what="counts")
            if total is not None and not _is_torch_cuda(total):
                raise TypeError("total: expected a torch CUDA int64 tensor of 2 elements")
            tptr = _ptr_and_flag(total, (8,), 2, what="total")[0]
            if asynchronous:
                flags |= ASYNC
            _check(self._lib.sieve_segment_counts(self._h, int(lo), int(hi), int(seg_width), cptr, nb, tptr, flags),
                   "sieve_segment_counts")
            return None
        if counts is None:
            counts = np.zeros(max(nb, 1), dtype=np.uint64)
        cptr = _ptr_and_flag(counts, (8,), nb, what="counts")[0]
        r = CountResult()
        _check(self._lib.sieve_segment_counts(self._h, int(lo), int(hi), int(seg_width), cptr, nb,
                                              ctypes.cast(ctypes.byref(r), _p), 0), "sieve_segment_counts")
        return CountAndSum(r.count, r.checksum), counts[:nb]


class Server:
    """Request loop with continuous batching on a Sieve context (sieve_server_*).

    While a server runs, make no other call on its context."""

    def __init__(self, sieve: Sieve, pool_bytes: int = 1 << 30, max_batch: int = 0, max_queue: int = 0,
                 batch_scratch_bytes: int = 0):
        self._lib = lib()
        self.sieve = sieve
        cfg = ServerConfig(int(pool_bytes), int(max_batch), int(max_queue), int(batch_scratch_bytes))
        h = _p()
        _check(self._lib.sieve_server_start(sieve.handle, ctypes.byref(cfg), ctypes.byref(h)), "sieve_server_start")
        self._h = h

    def submit(self, lo: int, hi: int, mode: int) -> int:
        """Admit one query and return its id (SieveError with ERR_BUSY on backpressure)."""
        rid = _u64(0)
        _check(self._lib.sieve_server_submit(self._h, int(lo), int(hi), int(mode), ctypes.byref(rid)),
               "sieve_server_submit")
        return int(rid.value)

    def try_submit(self, lo: int, hi: int, mode: int):
        """Like submit, but None instead of an exception when the server is busy."""
        rid = _u64(0)
        rc = self._lib.sieve_server_submit(self._h, int(lo), int(hi), int(mode), ctypes.byref(rid))
        if rc == ERR_BUSY:
            return None
        _check(rc, "sieve_server_submit")
        return int(rid.value)

    def poll(self, rid: int, out=None):
        """None while pending; else (CountAndSum, primes or None) and the
        request is released.  `out` (numpy uint64 or torch CUDA int64) receives
        a list-mode answer; without it a numpy array is returned."""
        r = CountResult()
        n = _sz(0)
        if out is not None:
            ptr, flags, cap = _ptr_and_flag(out, (8,), what="out")
            rc = self._lib.sieve_server_poll(self._h, int(rid), ctypes.cast(ctypes.byref(r), _p), ptr, cap,
                                             ctypes.byref(n), flags)
            if rc == PENDING:
                return None
            _check(rc, "sieve_server_poll")
            return CountAndSum(r.count, r.checksum), int(n.value)
        rc = self._lib.sieve_server_poll(self._h, int(rid), ctypes.cast(ctypes.byref(r), _p), None, 0,
                                         ctypes.byref(n), 0)
        if rc == PENDING:
            return None
        if rc == ERR_CAPACITY and n.value > 0:
            buf = np.empty(int(n.value), dtype=np.uint64)
            rc = self._lib.sieve_server_poll(self._h, int(rid), ctypes.cast(ctypes.byref(r), _p),
                                             buf.ctypes.data, buf.size, ctypes.byref(n), 0)
            _check(rc, "sieve_server_poll")
            return CountAndSum(r.count, r.checksum), buf
        _check(rc, "sieve_server_poll")
        return CountAndSum(r.count, r.checksum), None

    def next_done(self, timeout_us: int = 0):
        """Id of a finished request, or None if none finished within timeout_us."""
        rid = _u64(0)
        rc = self._lib.sieve_server_next_done(self._h, ctypes.byref(rid), int(timeout_us))
        if rc == PENDING:
            return None
        _check(rc, "sieve_server_next_done")
        return int(rid.value)

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(self._lib.sieve_server_get_stats(self._h, ctypes.byref(st), int(bool(reset))), "sieve_server_get_stats")
        return st.as_dict()

    def stop(self) -> None:
        if getattr(self, "_h", None):
            self._lib.sieve_server_stop(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
