"""Python binding of libsvb.so: argument marshalling only.

Each function has the name and argument order of its C counterpart in
``include/svb.h``; device buffers are passed as torch CUDA tensors (or raw
integer device addresses), sizes as ints.  Every computation runs in the
library's CUDA kernels; there is no host or PyTorch fallback, and importing
a function without the built library raises.

Synchronous calls run on torch's current CUDA stream (``svb_set_stream`` is
called with it before each call).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsvb.so")
ERROR = (1 << 64) - 1  # SVB_ERROR

SVB_OK, SVB_EINVAL, SVB_ETRUNCATED, SVB_ECUDA, SVB_ETIMEOUT, SVB_ENOMEM = range(6)


class SvbError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} (status {status})")


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libsvb.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        sz, u32, u64, i32, vp = (ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.c_int, ctypes.c_void_p)
        sig = {
            "svb_max_compressed_size": ([sz], sz),
            "svb_compressed_size_from_control": ([vp, sz], sz),
            "svb_encode": ([vp, sz, vp], sz),
            "svb_decode": ([vp, sz, vp], sz),
            "svb_delta_encode": ([vp, sz, vp, u32], sz),
            "svb_delta_decode": ([vp, sz, vp, u32], sz),
            "svb_decode_checked": ([vp, sz, sz, vp, u32, i32], sz),
            "svb_decode_host": ([vp, sz, sz, vp, u32, i32, vp, vp], sz),
            "svb_encode_host": ([vp, sz, vp, u32, i32, vp, vp], sz),
            "svb_set_stream": ([vp], i32),
            "svb_get_stream": ([], vp),
            "svb_last_error": ([], i32),
            "svb_error_string": ([i32], ctypes.c_char_p),
            "svb_set_spin_limit": ([u64], None),
            "svb_set_decode_variant": ([i32], i32),
            "svb_set_encode_variant": ([i32], i32),
            "svb_workspace_size": ([sz], sz),
            "svb_workspace_init": ([vp, sz, vp], i32),
            "svb_encode_async": ([vp, sz, vp, u32, i32, vp, vp, sz, vp], i32),
            "svb_decode_async": ([vp, sz, sz, vp, u32, i32, vp, vp, sz, vp], i32),
            "svb_testhook_lookback_timeout": ([vp, sz, vp, u64, vp, vp, sz, vp], i32),
            "svb_testhook_offsets_timeout": ([vp, sz, vp, u64, vp, vp, sz, vp], i32),
            "svb_decode_noalloc": ([vp, sz, sz, vp, u32, i32, vp], sz),
            "svb_query_batch": ([vp, sz, vp, i32, vp, sz, vp, vp], i32),
            "svb_append": ([vp, sz, vp, sz, sz, sz, vp, sz, u32, i32], sz),
            "svb_size_report": ([vp, sz, u32, i32, vp], i32),
            "svb_size_report_async": ([vp, sz, u32, i32, vp, vp], i32),
            "svb_batch_plan_bytes": ([sz], sz),
            "svb_profile_begin": ([], i32),
            "svb_profile_end": ([ctypes.c_char_p, sz], sz),
            "svb_batch_plan": ([vp, sz, u32, vp, sz, vp], i32),
            "svb_batch_plan_segments": ([vp, sz, u32, u32, vp, sz, vp], i32),
            "svb_batch_workspace_size": ([], sz),
            "svb_batch_set_stages": ([i32, i32], i32),
            "svb_batch_get_stages": ([i32], i32),
            "svb_batch_set_tile": ([i32], i32),
            "svb_batch_get_tile": ([], i32),
            "svb_batch_decode": ([vp, vp, vp, vp, i32, vp, vp, sz, i32, vp], i32),
            "svb_batch_encode": ([vp, vp, vp, vp, i32, vp, vp, vp, sz, i32, vp], i32),
            "svb_decode_each": ([vp, sz, vp, vp, i32, vp, vp, sz, vp], i32),
            "svb_control_range_bytes": ([vp, sz, sz, sz, vp, vp], i32),
            "svb_gap_sum": ([vp, sz, sz, vp, vp, sz, vp], i32),
            "svb_encode_each": ([vp, sz, vp, vp, i32, vp, vp, sz, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _p(x) -> int:
    """Device (or host) address of a tensor, array or integer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


def _stream(stream=None) -> int:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _sized(k: int, what: str) -> int:
    if k == ERROR:
        raise SvbError(lib().svb_last_error(), what)
    return k


def error_string(status: int) -> str:
    return lib().svb_error_string(status).decode()


def svb_max_compressed_size(n: int) -> int:
    return lib().svb_max_compressed_size(n)


def svb_compressed_size_from_control(h_ctrl, n: int) -> int:
    return _sized(lib().svb_compressed_size_from_control(_p(h_ctrl), n),
                  "svb_compressed_size_from_control")


def svb_encode(inp, n: int, out) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_encode(_p(inp), n, _p(out)), "svb_encode")


def svb_decode(inp, n: int, out) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_decode(_p(inp), n, _p(out)), "svb_decode")


def svb_delta_encode(inp, n: int, out, prev: int) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_delta_encode(_p(inp), n, _p(out), prev & 0xFFFFFFFF),
                  "svb_delta_encode")


def svb_delta_decode(inp, n: int, out, prev: int) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_delta_decode(_p(inp), n, _p(out), prev & 0xFFFFFFFF),
                  "svb_delta_decode")


def svb_decode_checked(inp, in_len: int, n: int, out, prev: int, delta: int) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_decode_checked(_p(inp), in_len, n, _p(out), prev & 0xFFFFFFFF,
                                           int(delta)), "svb_decode_checked")


def svb_decode_host(h_in, in_len: int, n: int, h_out, prev: int, delta: int, d_in, d_out) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_decode_host(_p(h_in), in_len, n, _p(h_out), prev & 0xFFFFFFFF,
                                        int(delta), _p(d_in), _p(d_out)), "svb_decode_host")


def svb_encode_host(h_in, n: int, h_out, prev: int, delta: int, d_in, d_out) -> int:
    lib().svb_set_stream(_stream())
    return _sized(lib().svb_encode_host(_p(h_in), n, _p(h_out), prev & 0xFFFFFFFF,
                                        int(delta), _p(d_in), _p(d_out)), "svb_encode_host")


def svb_set_spin_limit(iterations: int) -> None:
    lib().svb_set_spin_limit(iterations)


(SVB_DECODE_AUTO, SVB_DECODE_SINGLE_PASS, SVB_DECODE_TWO_PASS, SVB_DECODE_SUMS_PASS,
 SVB_DECODE_SMALL, SVB_DECODE_CHUNKED) = 0, 1, 2, 3, 4, 5


def svb_set_decode_variant(variant: int) -> int:
    return lib().svb_set_decode_variant(variant)


SVB_ENCODE_AUTO, SVB_ENCODE_TILE_LOOKBACK, SVB_ENCODE_CHUNKED, SVB_ENCODE_SMALL = 0, 1, 2, 3


def svb_set_encode_variant(variant: int) -> int:
    return lib().svb_set_encode_variant(variant)


def svb_last_error() -> int:
    return lib().svb_last_error()


def svb_workspace_size(n: int) -> int:
    return lib().svb_workspace_size(n)


def svb_workspace_init(ws, ws_bytes: int, stream=None) -> int:
    return lib().svb_workspace_init(_p(ws), ws_bytes, _stream(stream))


def svb_encode_async(inp, n, out, prev, delta, d_result, ws, ws_bytes, stream=None) -> int:
    return lib().svb_encode_async(_p(inp), n, _p(out), prev & 0xFFFFFFFF, int(delta),
                                  _p(d_result), _p(ws), ws_bytes, _stream(stream))


def svb_decode_async(inp, in_len, n, out, prev, delta, d_result, ws, ws_bytes, stream=None) -> int:
    return lib().svb_decode_async(_p(inp), in_len, n, _p(out), prev & 0xFFFFFFFF, int(delta),
                                  _p(d_result), _p(ws), ws_bytes, _stream(stream))


# numpy layout of struct svb_list (32 bytes)
def list_dtype():
    import numpy as np
    return np.dtype([("in_off", "<u8"), ("in_len", "<u8"), ("out_off", "<u8"),
                     ("n", "<u4"), ("prev", "<u4")])


def svb_batch_plan_bytes(num_lists: int) -> int:
    return lib().svb_batch_plan_bytes(num_lists)


def svb_batch_plan(h_lists, num_lists: int, big_threshold: int, d_plan, plan_bytes: int,
                   stream=None) -> int:
    return lib().svb_batch_plan(_p(h_lists), num_lists, big_threshold, _p(d_plan), plan_bytes,
                                _stream(stream))


def svb_batch_plan_segments(h_lists, num_lists: int, big_threshold: int, segment_tiles: int,
                            d_plan, plan_bytes: int, stream=None) -> int:
    return lib().svb_batch_plan_segments(_p(h_lists), num_lists, big_threshold, segment_tiles,
                                         _p(d_plan), plan_bytes, _stream(stream))


def svb_batch_set_stages(decode_stages: int, encode_stages: int) -> int:
    return lib().svb_batch_set_stages(decode_stages, encode_stages)


def svb_batch_get_stages(encode: int) -> int:
    return lib().svb_batch_get_stages(encode)


def svb_batch_set_tile(tile_ints: int) -> int:
    return lib().svb_batch_set_tile(tile_ints)


def svb_batch_get_tile() -> int:
    return lib().svb_batch_get_tile()


def svb_batch_workspace_size() -> int:
    return lib().svb_batch_workspace_size()


def svb_batch_decode(d_plan, d_lists, in_base, out_base, delta, d_result, ws, ws_bytes,
                     grid: int = 0, stream=None) -> int:
    return lib().svb_batch_decode(_p(d_plan), _p(d_lists), _p(in_base), _p(out_base), int(delta),
                                  _p(d_result), _p(ws), ws_bytes, grid, _stream(stream))


def svb_batch_encode(d_plan, d_lists, in_base, out_base, delta, d_sizes, d_result, ws, ws_bytes,
                     grid: int = 0, stream=None) -> int:
    return lib().svb_batch_encode(_p(d_plan), _p(d_lists), _p(in_base), _p(out_base), int(delta),
                                  _p(d_sizes), _p(d_result), _p(ws), ws_bytes, grid,
                                  _stream(stream))


def svb_decode_each(h_lists, num_lists, in_base, out_base, delta, d_results, ws, ws_bytes,
                    stream=None) -> int:
    return lib().svb_decode_each(_p(h_lists), num_lists, _p(in_base), _p(out_base), int(delta),
                                 _p(d_results), _p(ws), ws_bytes, _stream(stream))


def svb_encode_each(h_lists, num_lists, in_base, out_base, delta, d_results, ws, ws_bytes,
                    stream=None) -> int:
    return lib().svb_encode_each(_p(h_lists), num_lists, _p(in_base), _p(out_base), int(delta),
                                 _p(d_results), _p(ws), ws_bytes, _stream(stream))


def svb_control_range_bytes(in_, n, q0, q1, d_bytes, stream=None) -> int:
    return lib().svb_control_range_bytes(_p(in_), n, q0, q1, _p(d_bytes), _stream(stream))


def svb_gap_sum(in_, in_len, n, d_out, ws, ws_bytes, stream=None) -> int:
    return lib().svb_gap_sum(_p(in_), in_len, n, _p(d_out), _p(ws), ws_bytes, _stream(stream))


def svb_profile_begin() -> int:
    return lib().svb_profile_begin()


def svb_profile_end(buf=None, size: int = 0) -> int:
    return lib().svb_profile_end(buf, size)


def profile_end() -> dict:
    """Stop per-kernel timing: {kernel: (launches, total_ms)}."""
    buf = ctypes.create_string_buffer(1 << 16)  # one call: it consumes the records
    lib().svb_profile_end(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, count, ms = line.rsplit(" ", 2)
        out[name] = (int(count), float(ms))
    return out


SVB_NOALLOC_MAX_N = 1 << 24


def svb_append(ctrl, ctrl_cap: int, data, data_cap: int, data_len: int, n: int, inp, k: int,
               last: int, delta: int) -> int:
    return _sized(lib().svb_append(_p(ctrl), ctrl_cap, _p(data), data_cap, data_len, n, _p(inp),
                                   k, last & 0xFFFFFFFF, int(delta)), "svb_append")


SVB_SEEK, SVB_SELECT = 0, 1


def query_dtype():
    """numpy dtype laid out like svb_query."""
    import numpy as np
    return np.dtype([("list", np.uint32), ("op", np.uint32), ("arg", np.uint64)])


def answer_dtype():
    """numpy dtype laid out like svb_answer."""
    import numpy as np
    return np.dtype([("index", np.uint64), ("value", np.uint32), ("status", np.uint32)])


def svb_query_batch(d_lists, num_lists: int, in_base, delta: int, d_queries, num_queries: int,
                    d_answers, stream=None) -> int:
    return lib().svb_query_batch(_p(d_lists), num_lists, _p(in_base), int(delta), _p(d_queries),
                                 num_queries, _p(d_answers), _stream(stream))


def svb_size_report(inp, n: int, prev: int, delta: int, sizes) -> int:
    """sizes: a writable host buffer of two uint64 (numpy array)."""
    return lib().svb_size_report(_p(inp), n, prev & 0xFFFFFFFF, int(delta), _p(sizes))


def svb_size_report_async(inp, n: int, prev: int, delta: int, d_sizes, stream=None) -> int:
    return lib().svb_size_report_async(_p(inp), n, prev & 0xFFFFFFFF, int(delta), _p(d_sizes),
                                       _stream(stream))


def size_report(x, delta: bool = False, prev: int = 0) -> tuple[int, int]:
    """(Stream VByte bytes, VByte bytes) of a CUDA tensor of 4-byte integers."""
    import numpy as np
    sizes = np.zeros(2, dtype=np.uint64)
    st = svb_size_report(x, x.numel(), prev, int(delta), sizes)
    if st != 0:
        raise SvbError(st, "svb_size_report")
    return int(sizes[0]), int(sizes[1])


def svb_decode_noalloc(inp, in_len: int, n: int, out, prev: int, delta: int, stream=None) -> int:
    return _sized(lib().svb_decode_noalloc(_p(inp), in_len, n, _p(out), prev & 0xFFFFFFFF,
                                           int(delta), _stream(stream)), "svb_decode_noalloc")


def svb_testhook_lookback_timeout(stream_in, n, out, spin_limit, d_result, ws, ws_bytes,
                                  stream=None) -> int:
    return lib().svb_testhook_lookback_timeout(_p(stream_in), n, _p(out), spin_limit,
                                               _p(d_result), _p(ws), ws_bytes, _stream(stream))


def svb_testhook_offsets_timeout(stream_in, n, out, spin_limit, d_result, ws, ws_bytes,
                                 stream=None) -> int:
    return lib().svb_testhook_offsets_timeout(_p(stream_in), n, _p(out), spin_limit,
                                              _p(d_result), _p(ws), ws_bytes, _stream(stream))


# ---- tensor conveniences (allocation through torch, compute in the library) --

def encode(x, delta: bool = False, prev: int = 0):
    """Compressed stream (uint8 CUDA tensor, exact length) of a CUDA tensor of
    4-byte integers."""
    import torch
    n = x.numel()
    out = torch.empty(max(1, svb_max_compressed_size(n)), dtype=torch.uint8, device=x.device)
    if delta:
        k = svb_delta_encode(x, n, out, prev)
    else:
        k = svb_encode(x, n, out)
    return out[:k]


def decode(stream, n: int, delta: bool = False, prev: int = 0, checked: bool = True):
    """Decoded int32-typed CUDA tensor (the bits of the uint32 values)."""
    import torch
    out = torch.empty(max(1, n), dtype=torch.int32, device=stream.device)
    if checked:
        svb_decode_checked(stream, stream.numel(), n, out, prev, int(delta))
    elif delta:
        svb_delta_decode(stream, n, out, prev)
    else:
        svb_decode(stream, n, out)
    return out[:n]


def svb_error_string(status: int) -> str:
    return error_string(status)


def svb_set_stream(stream) -> int:
    return lib().svb_set_stream(_stream(stream))


def svb_get_stream() -> int:
    return lib().svb_get_stream() or 0
