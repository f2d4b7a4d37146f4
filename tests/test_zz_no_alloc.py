"""The entry point that allocates nothing (sieve_range_list_noalloc), called
through the C ABI, against the regular list call (sieve_range in list mode):
exact equality, on two calls in a row that share the fixed scratch array.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

from paper_2310_17746_gb300 import binding

pytestmark = pytest.mark.gpu


def test_no_alloc_list_matches_regular_list():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with binding.Sieve(10**12 + 10**8) as sv:
        # two calls in a row: a wide range near 1e12, then a narrower one from 0 whose
        # tiles reuse (and must overwrite) what the first call left in the scratch
        for lo, hi in ((10**12 - 50_000_000, 10**12 + 40_000_000), (0, 3_000_000)):
            want = sv.range_list(lo, hi)
            ref = sv.range_count(lo, hi)
            out = torch.full((want.size + 64,), -1, dtype=torch.int64, device="cuda")
            n, cs = sv.range_list_noalloc(lo, hi, out)
            torch.cuda.synchronize()
            assert n == want.size
            assert (cs.count, cs.checksum) == (ref.count, ref.checksum)
            got = out[:n].cpu().numpy().astype(np.uint64)
            assert np.array_equal(got, want)
            assert int(out[n]) == -1  # nothing written past the list


def test_no_alloc_rejects_ranges_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with binding.Sieve(10**12) as sv:
        out = torch.zeros(16, dtype=torch.int64, device="cuda")
        with pytest.raises(binding.SieveError) as e:
            sv.range_list_noalloc(0, 10**10, out)
        assert e.value.status == binding.ERR_INVALID
        assert "scratch" in binding.last_error()
        with pytest.raises(binding.SieveError) as e:
            sv.range_list_noalloc(0, 1000, out)  # 168 primes do not fit in 16 slots
        assert e.value.status == binding.ERR_CAPACITY
