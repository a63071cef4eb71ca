"""Argument checks of the C ABI that return before any CUDA call, run on a
machine without a GPU: null pointers, short inputs, undersized workspaces,
unknown variants, and the empty call.  Device addresses passed here are
placeholders that the checks reject before anything could dereference them."""
from __future__ import annotations

import ctypes

import pytest

from paper_1709_08990_gb300 import _build, svb

FAKE = ctypes.c_void_p(0x1000)  # never dereferenced: every call below returns first


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return svb.lib()


def test_null_buffers_give_einval(lib):
    for f in (lib.svb_encode, lib.svb_decode):
        assert f(None, 10, None) == svb.ERROR
        assert lib.svb_last_error() == svb.SVB_EINVAL
    assert lib.svb_delta_encode(None, 10, None, 0) == svb.ERROR
    assert lib.svb_delta_decode(None, 10, None, 0) == svb.ERROR
    assert lib.svb_decode_checked(None, 100, 10, None, 0, 1) == svb.ERROR
    assert lib.svb_last_error() == svb.SVB_EINVAL
    assert lib.svb_decode_host(None, 100, 10, None, 0, 0, None, None) == svb.ERROR
    assert lib.svb_encode_host(None, 10, None, 0, 0, None, None) == svb.ERROR
    assert lib.svb_last_error() == svb.SVB_EINVAL


def test_empty_calls_return_zero_and_ok(lib):
    assert lib.svb_encode(None, 0, None) == 0
    assert lib.svb_decode(None, 0, None) == 0
    assert lib.svb_decode_checked(None, 0, 0, None, 0, 0) == 0
    assert lib.svb_last_error() == svb.SVB_OK


def test_input_shorter_than_its_control_bytes_is_truncated(lib):
    n = 1000  # needs 250 control bytes
    assert lib.svb_decode_checked(FAKE, 249, n, FAKE, 0, 0) == svb.ERROR
    assert lib.svb_last_error() == svb.SVB_ETRUNCATED
    ws = lib.svb_workspace_size(n)
    st = lib.svb_decode_async(FAKE, 100, n, FAKE, 0, 1, FAKE, FAKE, ws, None)
    assert st == svb.SVB_ETRUNCATED


def test_async_forms_check_result_and_workspace(lib):
    n = 1 << 20
    ws = lib.svb_workspace_size(n)
    assert lib.svb_encode_async(FAKE, n, FAKE, 0, 0, None, FAKE, ws, None) == svb.SVB_EINVAL
    assert lib.svb_decode_async(FAKE, 5 * n, n, FAKE, 0, 0, None, FAKE, ws, None) == \
        svb.SVB_EINVAL
    assert lib.svb_encode_async(FAKE, n, FAKE, 0, 0, FAKE, FAKE, ws - 1, None) == svb.SVB_EINVAL
    assert lib.svb_decode_async(FAKE, 5 * n, n, FAKE, 0, 0, FAKE, FAKE, ws - 1, None) == \
        svb.SVB_EINVAL
    assert lib.svb_encode_async(None, n, FAKE, 0, 0, FAKE, FAKE, ws, None) == svb.SVB_EINVAL
    assert lib.svb_workspace_init(None, ws, None) == svb.SVB_EINVAL


def test_workspace_size_grows_with_n(lib):
    sizes = [lib.svb_workspace_size(n) for n in (1, 512, 4096, 65536, 1 << 20, 1 << 30)]
    assert all(a <= b for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] > sizes[0]
    plans = [lib.svb_batch_plan_bytes(k) for k in (1, 10, 1000, 100_000)]
    assert all(a < b for a, b in zip(plans, plans[1:]))


def test_variants_reject_unknown_values(lib):
    for v in (-1, 6, 99):
        assert lib.svb_set_decode_variant(v) == svb.SVB_EINVAL
    for v in (-1, 4):
        assert lib.svb_set_encode_variant(v) == svb.SVB_EINVAL
    try:
        for v in (0, 1, 2, 3, 4, 5):
            assert lib.svb_set_decode_variant(v) == svb.SVB_OK
        for v in (0, 1, 2, 3):
            assert lib.svb_set_encode_variant(v) == svb.SVB_OK
    finally:
        lib.svb_set_decode_variant(0)
        lib.svb_set_encode_variant(0)


def test_test_hooks_reject_bad_arguments(lib):
    n = 3 * 65536 + 5
    ws = lib.svb_workspace_size(n)
    assert lib.svb_testhook_offsets_timeout(FAKE, 65536, FAKE, 10, FAKE, FAKE,
                                            lib.svb_workspace_size(65536), None) == svb.SVB_EINVAL
    assert lib.svb_testhook_offsets_timeout(None, n, FAKE, 10, FAKE, FAKE, ws, None) == \
        svb.SVB_EINVAL
    assert lib.svb_testhook_offsets_timeout(FAKE, n, FAKE, 10, FAKE, FAKE, ws - 1, None) == \
        svb.SVB_EINVAL
    assert lib.svb_testhook_lookback_timeout(FAKE, 100, FAKE, 10, FAKE, FAKE,
                                             lib.svb_workspace_size(100), None) == svb.SVB_EINVAL
