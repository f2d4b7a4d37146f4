"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares; the Python binding covers each of them."""
import glob
import os
import re

from paper_2310_17746_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sieve_[A-Za-z0-9_]+)\s*\(", re.M)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(DECL.findall(text))
    return sorted(names)


def test_header_declares_the_calls():
    names = declared_functions()
    for must in ("sieve_create", "sieve_destroy", "sieve_count", "sieve_primes", "sieve_range",
                 "sieve_segment_counts", "sieve_last_error", "sieve_range_batch", "sieve_range_each",
                 "sieve_autotune_batch", "sieve_autotune_range", "sieve_server_start", "sieve_server_submit",
                 "sieve_server_poll", "sieve_server_next_done", "sieve_server_get_stats", "sieve_server_stop"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = binding.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if n not in binding.SIGNATURES]
    assert not missing, missing


def test_no_cpu_fallback_without_gpu():
    """With no CUDA device the library refuses to create a context (no CPU path)."""
    import torch
    if torch.cuda.is_available():
        return
    try:
        binding.Sieve(10**6)
    except binding.SieveError as e:
        assert e.status in (binding.ERR_CUDA, binding.ERR_INVALID)
    else:
        raise AssertionError("a context was created without a GPU")
