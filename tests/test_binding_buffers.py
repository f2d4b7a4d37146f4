"""The binding rejects output buffers that the library could overrun, before
any library call: wrong element size or type, non-contiguous views (e.g. a
stride-0 expand), too few elements for a fixed-size output, read-only host
arrays.  Runs on the CPU: the device buffers are stand-ins with the attributes
the binding reads, and the library handle is a recorder that fails the test if
it is ever called."""
import numpy as np
import pytest

from paper_2310_17746_gb300 import binding


class FakeDeviceTensor:
    """What the binding reads from a torch CUDA tensor, nothing more."""

    def __init__(self, dtype: str, numel: int, esize: int, contiguous: bool = True):
        self.is_cuda = True
        self.dtype = dtype
        self._n, self._e, self._c = numel, esize, contiguous

    def element_size(self):
        return self._e

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x10000


class NoCalls:
    def __getattr__(self, name):
        raise AssertionError(f"library function {name} was called with a bad buffer")


@pytest.fixture
def sv():
    s = object.__new__(binding.Sieve)
    s._lib = NoCalls()
    s._h = None
    s.device = 0
    s.max_hi = 10**12
    return s


def test_list_rejects_wrong_element_type(sv):
    with pytest.raises(TypeError):
        sv.range_list(0, 1000, out=FakeDeviceTensor("torch.int32", 1000, 4))
    with pytest.raises(TypeError):
        sv.range_list(0, 1000, out=FakeDeviceTensor("torch.uint8", 8000, 1))
    with pytest.raises(TypeError):
        sv.range_list(0, 1000, out=np.zeros(100, dtype=np.float64))
    with pytest.raises(TypeError):
        sv.range_list(0, 1000, out=np.zeros(100, dtype=np.uint32))


def test_list_rejects_non_contiguous_and_read_only(sv):
    with pytest.raises(ValueError):
        sv.range_list(0, 1000, out=FakeDeviceTensor("torch.int64", 1000, 8, contiguous=False))
    a = np.zeros(100, dtype=np.uint64)
    a.flags.writeable = False
    with pytest.raises(ValueError):
        sv.range_list(0, 1000, out=a)
    with pytest.raises(ValueError):
        sv.range_list(0, 1000, out=np.zeros(200, dtype=np.uint64)[::2])


def test_count_out_needs_two_int64(sv):
    with pytest.raises(ValueError):
        sv.range_count(0, 1000, out=FakeDeviceTensor("torch.int64", 1, 8))
    with pytest.raises(TypeError):
        sv.range_count(0, 1000, out=FakeDeviceTensor("torch.int32", 4, 4))
    with pytest.raises(TypeError):
        sv.range_count(0, 1000, out=np.zeros(2, dtype=np.uint64))  # host memory is not a device pointer


def test_noalloc_and_next_and_primes(sv):
    with pytest.raises(TypeError):
        sv.range_list_noalloc(0, 1000, FakeDeviceTensor("torch.int32", 1000, 4))
    with pytest.raises(ValueError):
        sv.range_list_noalloc(0, 1000, FakeDeviceTensor("torch.int64", 1000, 8, contiguous=False))
    with pytest.raises(TypeError):
        sv.next_primes(10, 5, out=FakeDeviceTensor("torch.int32", 5, 4))
    with pytest.raises(TypeError):
        sv.primes(100, out=FakeDeviceTensor("torch.int16", 100, 2))


def test_segment_counts_and_batch_sizes(sv):
    with pytest.raises(ValueError):  # 3 bins needed
        sv.segment_counts(0, 3 * 6144, 6144, counts=np.zeros(2, dtype=np.uint64))
    with pytest.raises(ValueError):
        sv.segment_counts(0, 3 * 6144, 6144, counts=FakeDeviceTensor("torch.int64", 2, 8),
                          total=FakeDeviceTensor("torch.int64", 2, 8))
    with pytest.raises(ValueError):
        sv.segment_counts(0, 3 * 6144, 6144, counts=FakeDeviceTensor("torch.int64", 3, 8),
                          total=FakeDeviceTensor("torch.int64", 1, 8))
    lo, hi, mode = [0, 10], [5, 20], [0, 1]
    with pytest.raises(ValueError):  # cnt needs 2 * nq
        sv.range_batch(lo, hi, mode, cnt=FakeDeviceTensor("torch.int64", 3, 8),
                       offsets=FakeDeviceTensor("torch.int64", 3, 8), values=FakeDeviceTensor("torch.int64", 9, 8))
    with pytest.raises(ValueError):  # offsets need nq + 1
        sv.range_batch(lo, hi, mode, cnt=np.zeros((2, 2), np.uint64), offsets=np.zeros(2, np.uint64))
    with pytest.raises(TypeError):
        sv.range_batch(lo, hi, mode, cnt=FakeDeviceTensor("torch.int64", 4, 8),
                       offsets=FakeDeviceTensor("torch.int64", 3, 8), values=FakeDeviceTensor("torch.int32", 9, 4))
