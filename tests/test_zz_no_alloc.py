"""svb_decode_noalloc against svb_decode_checked, through the C ABI.

svb_decode_noalloc serves callers that cannot allocate device memory while
they decode (an allocator decoding inside its own bookkeeping, a process whose
HBM a caching allocator already holds, a path that cannot afford the device
synchronisation cudaMalloc/cudaFree may cause).  It decodes with a fixed
scratch array inside the library.  Its results must equal those of the
regular entry point, bit for bit (the codec is integer arithmetic), on two
calls in a row, since every call reuses the same scratch.  This file is
collected last so that a failure here leaves every other test already run.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1709_08990_gb300 import svb
from paper_1709_08990_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _decode_both(stream_bytes, n, delta, prev):
    lib = svb.lib()
    got = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    want = torch.full((n,), -2, dtype=torch.int32, device=DEV)
    k_new = lib.svb_decode_noalloc(stream_bytes.data_ptr(), stream_bytes.numel(), n,
                                   got.data_ptr(), prev, int(delta), _stream())
    assert k_new != svb.ERROR, svb.error_string(lib.svb_last_error())
    k_old = svb.svb_decode_checked(stream_bytes, stream_bytes.numel(), n, want, prev, int(delta))
    return k_new, k_old, got, want


def test_noalloc_decode_matches_checked_decode_twice():
    cases = [
        (W.skewed_lengths(31, 3_000_001), False, 0),             # several tiles, ragged tail
        (W.sorted_geometric(32, 2_500_003, 16.0, 7), True, 7),   # differential, start 7
    ]
    for values, delta, prev in cases:
        x = torch.from_numpy(values.view(np.int32)).to(DEV)
        s = svb.encode(x, delta=delta, prev=prev)
        for _ in range(2):  # the second call reuses the scratch the first left behind
            k_new, k_old, got, want = _decode_both(s, values.size, delta, prev)
            assert k_new == k_old == s.numel()
            assert torch.equal(got, want)
            assert torch.equal(got, x)


def test_noalloc_at_its_limit_then_smaller():
    """n at the limit fills the scratch exactly; the calls after it, of other
    sizes, find their tile records where the large call left offsets and
    carries.  Each must still equal svb_decode_checked and the values."""
    n_max = svb.SVB_NOALLOC_MAX_N
    cases = [
        (W.skewed_lengths(33, n_max), False, 0),
        (W.sorted_geometric(34, 1 << 18, 16.0, 3), True, 3),
        (W.skewed_lengths(35, (1 << 18) + 1), False, 0),
        (W.sorted_geometric(36, n_max, 16.0, 0), True, 0),
        (W.skewed_lengths(37, 777_777), True, 99),
    ]
    for values, delta, prev in cases:
        x = torch.from_numpy(values.view(np.int32)).to(DEV)
        s = svb.encode(x, delta=delta, prev=prev)
        k_new, k_old, got, want = _decode_both(s, values.size, delta, prev)
        assert k_new == k_old == s.numel()
        assert torch.equal(got, want)
        assert torch.equal(got, x)


def test_noalloc_empty_call_clears_the_last_error():
    lib = svb.lib()
    dummy = torch.zeros(16, dtype=torch.uint8, device=DEV)
    k = lib.svb_decode_noalloc(dummy.data_ptr(), 16, svb.SVB_NOALLOC_MAX_N + 1,
                               dummy.data_ptr(), 0, 0, _stream())
    assert k == svb.ERROR and lib.svb_last_error() == svb.SVB_EINVAL
    assert lib.svb_decode_noalloc(dummy.data_ptr(), 16, 0, dummy.data_ptr(), 0, 0, _stream()) == 0
    assert lib.svb_last_error() == svb.SVB_OK


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = svb.lib()
    n = svb.SVB_NOALLOC_MAX_N + 1
    dummy = torch.zeros(16, dtype=torch.uint8, device=DEV)
    k = lib.svb_decode_noalloc(dummy.data_ptr(), ctypes.c_size_t(-1).value, n,
                               dummy.data_ptr(), 0, 0, _stream())
    assert k == svb.ERROR
    assert lib.svb_last_error() == svb.SVB_EINVAL
