"""Stream VByte oracle (test infrastructure only).

A plain scalar C statement of the codec in ``svb_ref.c`` (arXiv 1709.08990,
Sec. 3-4 for the format, Sec. 1, 2 and 5 for differential coding), wrapped
here with ctypes over numpy arrays.  Only the test suite, the smoke check
and the bench's CPU-baseline leg may import this package.  The product
library neither links nor calls it, and it shares no code with the CUDA
path.

Every function here is pinned by the ``-m "not gpu"`` tests: the paper's
worked byte examples (Fig. 1, Fig. 3), its prefix-sum example (Sec. 2), the
length boundaries (Sec. 3), the size formula (Sec. 4), brute force over all
length patterns for n <= 12, and an independently written Python definition.

``vbyte_ref.c`` (the ``VByte`` class) states the VByte format the paper
compares Stream VByte with (Sec. 2-3), for the size comparison of Sec. 5
(Fig. 5b); its pins are the paper's two byte examples (32, 128), the 7-bit
length boundaries, the decoding sum of Sec. 3 and the Python definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "svb_ref.c")
LIB = os.path.join(HERE, "libsvb_ref.so")

VSRC = os.path.join(HERE, "vbyte_ref.c")
VLIB = os.path.join(HERE, "libvbyte_ref.so")

PSRC = os.path.join(HERE, "par_ref.c")
PLIB = os.path.join(HERE, "libpar_ref.so")

ERROR = (1 << 64) - 1  # SVB_REF_ERROR, (size_t)-1


def build_cmd(src: str = SRC, out: str = LIB) -> list[str]:
    """gcc command that builds the oracle's shared library."""
    return ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", out, src]


def build() -> None:
    """Compile the oracle libraries that are missing or older than their source."""
    for src, lib in ((SRC, LIB), (VSRC, VLIB)):
        if os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
            continue
        subprocess.run(build_cmd(src, lib), check=True)
    # The multi-threaded timing harness links the oracle's own source.
    if not (os.path.exists(PLIB) and os.path.getmtime(PLIB) >= max(
            os.path.getmtime(PSRC), os.path.getmtime(SRC))):
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", PLIB,
                        PSRC, SRC], check=True)


class Codec:
    """The oracle's entry points, bound to one build of ``svb_ref.c``."""

    def __init__(self, path: str = LIB):
        L = ctypes.CDLL(path)
        sz, u32, vp = ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p
        L.svb_ref_byte_length.argtypes = [u32]
        L.svb_ref_byte_length.restype = ctypes.c_uint
        L.svb_ref_control_bytes.argtypes = [sz]
        L.svb_ref_control_bytes.restype = sz
        L.svb_ref_max_compressed_size.argtypes = [sz]
        L.svb_ref_max_compressed_size.restype = sz
        L.svb_ref_encode.argtypes = [vp, sz, vp]
        L.svb_ref_encode.restype = sz
        L.svb_ref_delta_encode.argtypes = [vp, sz, vp, u32]
        L.svb_ref_delta_encode.restype = sz
        L.svb_ref_decode.argtypes = [vp, sz, sz, vp]
        L.svb_ref_decode.restype = sz
        L.svb_ref_delta_decode.argtypes = [vp, sz, sz, vp, u32]
        L.svb_ref_delta_decode.restype = sz
        L.svb_ref_data_bytes.argtypes = [vp, sz]
        L.svb_ref_data_bytes.restype = sz
        L.svb_ref_seek.argtypes = [vp, sz, sz, u32, ctypes.c_int, u32, ctypes.POINTER(u32)]
        L.svb_ref_seek.restype = sz
        L.svb_ref_select.argtypes = [vp, sz, sz, u32, ctypes.c_int, sz, ctypes.POINTER(u32)]
        L.svb_ref_select.restype = sz
        self.lib = L
        self.path = path

    def byte_length(self, x: int) -> int:
        return self.lib.svb_ref_byte_length(x)

    def control_bytes(self, n: int) -> int:
        return self.lib.svb_ref_control_bytes(n)

    def max_compressed_size(self, n: int) -> int:
        return self.lib.svb_ref_max_compressed_size(n)

    def encode(self, x, prev: int = 0, delta: bool = False) -> np.ndarray:
        """Compressed stream (uint8) of the uint32 array ``x``."""
        x = np.ascontiguousarray(x, dtype=np.uint32)
        n = x.size
        # Room for n // 4 + 1 control bytes and four bytes per integer,
        # sized here rather than by max_compressed_size, which the pins test.
        out = np.zeros(n // 4 + 1 + 4 * n, dtype=np.uint8)
        if delta:
            k = self.lib.svb_ref_delta_encode(x.ctypes.data, n, out.ctypes.data,
                                              prev & 0xFFFFFFFF)
        else:
            k = self.lib.svb_ref_encode(x.ctypes.data, n, out.ctypes.data)
        if k == ERROR:
            raise MemoryError("oracle encode failed")
        return out[:k].copy()

    def decode(self, stream, n: int, prev: int = 0, delta: bool = False,
               in_len: int | None = None):
        """(decoded uint32 array, bytes consumed).  Bytes consumed is ERROR
        when the stream is shorter than its control bytes require."""
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        if in_len is None:
            in_len = stream.size
        assert in_len <= stream.size
        buf = stream if stream.size else np.zeros(1, dtype=np.uint8)
        out = np.zeros(max(1, n), dtype=np.uint32)
        if delta:
            k = self.lib.svb_ref_delta_decode(buf.ctypes.data, in_len, n,
                                              out.ctypes.data, prev & 0xFFFFFFFF)
        else:
            k = self.lib.svb_ref_decode(buf.ctypes.data, in_len, n, out.ctypes.data)
        return out[:n], k

    def seek(self, stream, n: int, target: int, prev: int = 0, delta: bool = False,
             in_len: int | None = None) -> tuple[int, int]:
        """(index of the first integer >= target or n, that integer or 0);
        index is ERROR when the stream ends before the answer is decided."""
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        buf = stream if stream.size else np.zeros(1, dtype=np.uint8)
        v = ctypes.c_uint32(0)
        k = self.lib.svb_ref_seek(buf.ctypes.data, stream.size if in_len is None else in_len,
                                  n, prev & 0xFFFFFFFF, int(delta), target & 0xFFFFFFFF,
                                  ctypes.byref(v))
        return k, v.value

    def select(self, stream, n: int, index: int, prev: int = 0, delta: bool = False,
               in_len: int | None = None) -> int | None:
        """The integer at `index`, or None when index >= n or the stream ends
        before it."""
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        buf = stream if stream.size else np.zeros(1, dtype=np.uint8)
        v = ctypes.c_uint32(0)
        k = self.lib.svb_ref_select(buf.ctypes.data, stream.size if in_len is None else in_len,
                                    n, prev & 0xFFFFFFFF, int(delta), index, ctypes.byref(v))
        return None if k == ERROR else v.value

    def data_bytes(self, ctrl, n: int) -> int:
        ctrl = np.ascontiguousarray(ctrl, dtype=np.uint8)
        return self.lib.svb_ref_data_bytes(ctrl.ctypes.data, n)


class VByte:
    """The VByte oracle's entry points, bound to one build of ``vbyte_ref.c``."""

    def __init__(self, path: str = VLIB):
        L = ctypes.CDLL(path)
        sz, u32, vp, i32 = ctypes.c_size_t, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
        L.vbyte_ref_length.argtypes = [u32]
        L.vbyte_ref_length.restype = ctypes.c_uint
        L.vbyte_ref_size.argtypes = [vp, sz, i32, u32]
        L.vbyte_ref_size.restype = sz
        L.vbyte_ref_encode.argtypes = [vp, sz, vp, i32, u32]
        L.vbyte_ref_encode.restype = sz
        L.vbyte_ref_decode.argtypes = [vp, sz, sz, vp, i32, u32]
        L.vbyte_ref_decode.restype = sz
        self.lib = L
        self.path = path

    def length(self, v: int) -> int:
        return self.lib.vbyte_ref_length(v & 0xFFFFFFFF)

    def size(self, x, prev: int = 0, delta: bool = False) -> int:
        x = np.ascontiguousarray(x, dtype=np.uint32)
        buf = x if x.size else np.zeros(1, dtype=np.uint32)
        return self.lib.vbyte_ref_size(buf.ctypes.data, x.size, int(delta), prev & 0xFFFFFFFF)

    def encode(self, x, prev: int = 0, delta: bool = False) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint32)
        buf = x if x.size else np.zeros(1, dtype=np.uint32)
        out = np.zeros(max(1, 5 * x.size), dtype=np.uint8)
        k = self.lib.vbyte_ref_encode(buf.ctypes.data, x.size, out.ctypes.data, int(delta),
                                      prev & 0xFFFFFFFF)
        return out[:k].copy()

    def decode(self, stream, n: int, prev: int = 0, delta: bool = False):
        """(decoded uint32 array, bytes consumed or ERROR)."""
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        buf = stream if stream.size else np.zeros(1, dtype=np.uint8)
        out = np.zeros(max(1, n), dtype=np.uint32)
        k = self.lib.vbyte_ref_decode(buf.ctypes.data, stream.size, n, out.ctypes.data,
                                      int(delta), prev & 0xFFFFFFFF)
        return out[:n], k


class Parallel:
    """The oracle's decoder run on several host threads (``par_ref.c``): a
    timing harness whose every byte count and integer comes from the oracle."""

    def __init__(self, path: str = PLIB):
        L = ctypes.CDLL(path)
        sz, vp = ctypes.c_size_t, ctypes.c_void_p
        L.svb_par_decode.argtypes = [vp, sz, sz, vp, ctypes.c_uint32, ctypes.c_int, ctypes.c_int]
        L.svb_par_decode.restype = sz
        self.lib = L

    def decode(self, stream, n: int, prev: int = 0, delta: bool = False, threads: int = 1,
               out=None):
        """(decoded uint32 array, bytes consumed or ERROR)."""
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        buf = stream if stream.size else np.zeros(1, dtype=np.uint8)
        if out is None:
            out = np.zeros(max(1, n), dtype=np.uint32)
        k = self.lib.svb_par_decode(buf.ctypes.data, stream.size, n, out.ctypes.data,
                                    prev & 0xFFFFFFFF, int(delta), threads)
        return out[:n], k


_default: Codec | None = None
_vbyte: VByte | None = None
_par: Parallel | None = None


def parallel() -> Parallel:
    global _par
    if _par is None:
        build()
        _par = Parallel(PLIB)
    return _par


def vbyte() -> VByte:
    global _vbyte
    if _vbyte is None:
        build()
        _vbyte = VByte(VLIB)
    return _vbyte


def codec() -> Codec:
    global _default
    if _default is None:
        build()
        _default = Codec(LIB)
    return _default


def encode(x, prev: int = 0, delta: bool = False) -> np.ndarray:
    return codec().encode(x, prev, delta)


def decode(stream, n: int, prev: int = 0, delta: bool = False, in_len: int | None = None):
    return codec().decode(stream, n, prev, delta, in_len)


def byte_length(x: int) -> int:
    return codec().byte_length(x)


def control_bytes(n: int) -> int:
    return codec().control_bytes(n)


def max_compressed_size(n: int) -> int:
    return codec().max_compressed_size(n)


def data_bytes(ctrl, n: int) -> int:
    return codec().data_bytes(ctrl, n)
