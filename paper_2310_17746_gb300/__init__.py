"""GB300-native segmented prime sieve (6k+1 / 6k+5 residue bitmaps).

The compute path is the C-ABI library built from csrc/ (CUDA for sm_103a);
`binding` is its thin ctypes layer.  Importing the package does not load the
library; the first call that needs it builds (if stale) and loads it, and
raises if that fails -- there is no CPU fallback.
"""
from __future__ import annotations

from .binding import (ASYNC, COUNT, LIST, OUT_DEVICE, CountAndSum, Server, Sieve, SieveError, last_error,
                      lib, table1_start)

__all__ = ["Sieve", "Server", "SieveError", "CountAndSum", "COUNT", "LIST", "OUT_DEVICE", "ASYNC",
           "lib", "last_error", "table1_start", "workloads", "shard"]
