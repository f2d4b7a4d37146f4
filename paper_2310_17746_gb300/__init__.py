"""GB300-native segmented prime sieve (6k+1 / 6k+5 residue bitmaps).

The compute path is the C-ABI library built from csrc/ (CUDA for sm_103a);
this package is its thin ctypes binding.  Importing the package does not load
the library; the first call that needs it does, and raises if it is missing.
"""
from __future__ import annotations

__all__ = ["workloads"]
