"""A second, independently written definition of Stream VByte for tiny inputs.

It states the format differently from the C oracle so that a slip in one is
unlikely to be repeated in the other:
  * the byte length comes from Python's ``int.bit_length`` (Sec. 3: an integer
    x needs ceil(log_256(x + 1)) bytes; zero still takes one byte);
  * the control stream is one little-endian integer in which integer i owns
    bits 2i..2i+1 (Sec. 4, Fig. 3: ceil(2N/8) control bytes, first integer in
    the low bits);
  * values are cut with ``int.to_bytes(..., "little")`` (Sec. 2: the shuffle
    keeps the low-order bytes of each 32-bit lane).
Differential coding (Sec. 1, Sec. 5) uses the gaps x_i - x_{i-1} mod 2^32 with
x_0 = prev; decoding is the running sum (Sec. 2).
Pure-Python loops: use it only for small n.
"""
from __future__ import annotations

from itertools import accumulate

M32 = (1 << 32) - 1


def length_of(v: int) -> int:
    return max(1, (v.bit_length() + 7) // 8)


def encode(xs: list[int], prev: int = 0, delta: bool = False) -> bytes:
    if delta:
        before = [prev] + list(xs[:-1])
        vals = [(x - p) & M32 for x, p in zip(xs, before)]
    else:
        vals = [x & M32 for x in xs]
    n = len(vals)
    bits = 0
    for i, v in enumerate(vals):
        bits |= (length_of(v) - 1) << (2 * i)
    ctrl = bits.to_bytes((2 * n + 7) // 8, "little")
    data = b"".join(v.to_bytes(length_of(v), "little") for v in vals)
    return ctrl + data


def decode(stream: bytes, n: int, prev: int = 0, delta: bool = False):
    """(values, bytes consumed) or (None, None) when the stream is too short."""
    nctrl = (2 * n + 7) // 8
    if len(stream) < nctrl:
        return None, None
    bits = int.from_bytes(stream[:nctrl], "little")
    pos = nctrl
    vals = []
    for i in range(n):
        ln = ((bits >> (2 * i)) & 3) + 1
        if pos + ln > len(stream):
            return None, None
        vals.append(int.from_bytes(stream[pos:pos + ln], "little"))
        pos += ln
    if delta:
        vals = [(prev + s) & M32 for s in accumulate(vals)]
    return vals, pos


# --- VByte (Sec. 2-3), stated with divmod by 128 and bit_length -------------

def vbyte_length(v: int) -> int:
    """Sec. 3: an integer in [2^(7(L-1)), 2^(7L)) takes L bytes; zero one."""
    return max(1, -(-v.bit_length() // 7))


def vbyte_encode(xs: list[int], prev: int = 0, delta: bool = False) -> bytes:
    """Sec. 2: seven bits per byte from the least significant end; a byte's
    top bit says that the next byte continues the integer."""
    if delta:
        before = [prev] + list(xs[:-1])
        vals = [(x - p) & M32 for x, p in zip(xs, before)]
    else:
        vals = [x & M32 for x in xs]
    out = bytearray()
    for v in vals:
        while True:
            v, group = divmod(v, 128)
            out.append(group + (128 if v else 0))
            if not v:
                break
    return bytes(out)


def vbyte_decode(stream: bytes, n: int, prev: int = 0, delta: bool = False) -> list[int]:
    """Sec. 3: the value is the sum of (b_i mod 2^7) * 2^(7i) over its bytes,
    the last of which is below 2^7."""
    vals, i = [], 0
    for _ in range(n):
        parts = []
        while True:
            b = stream[i]
            i += 1
            parts.append(b % 128)
            if b < 128:
                break
        vals.append(sum(p * 128 ** k for k, p in enumerate(parts)) & M32)
    if delta:
        return [(prev + s) & M32 for s in accumulate(vals)]
    return vals
