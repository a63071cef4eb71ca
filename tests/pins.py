"""Checks that tie a build of the oracle to what the paper fixes.

Each function takes an ``oracle.Codec`` and returns a list of failure
messages (empty when the build agrees with the paper).  The same checks run
against the real oracle, where they must all pass, and against copies of the
oracle with a mistake planted on purpose, where at least one must fail.
"""
from __future__ import annotations

import os

import numpy as np

import svb_definition as D

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_golden(name: str) -> dict[str, list[str]]:
    out: dict[str, list[str]] = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            out.setdefault(key.strip(), []).append(val.strip())
    return out


def fig3_stream(c) -> list[str]:
    """Fig. 3 (Sec. 4): the exact 15 bytes of 1024,12,10,2^30,1,2,3,1024."""
    g = _read_golden("fig3_stream.txt")
    vals = [int(v) for v in g["values"][0].split()]
    want = bytes(int(b, 16) for b in g["stream"][0].split())
    errs = []
    got = c.encode(np.array(vals, dtype=np.uint32)).tobytes()
    if got != want:
        errs.append(f"fig3 encode {got.hex()} != {want.hex()}")
    back, k = c.decode(np.frombuffer(want, dtype=np.uint8), len(vals))
    if k != len(want) or back.tolist() != vals:
        errs.append(f"fig3 decode {back.tolist()} consumed {k}")
    rejected = bytes(int(b, 16) for b in g["rejected_msb_first_ctrl"][0].split())
    if got[:2] == rejected:
        errs.append("fig3 control bytes follow the rejected MSB-first reading")
    return errs


def fig1_blocks(c) -> list[str]:
    """Fig. 1 (Sec. 3): one block of four takes 9 resp. 6 bytes."""
    g = _read_golden("fig1_blocks.txt")
    errs = []
    for blk, nb in zip(g["block"], g["bytes"]):
        vals = np.array([int(v) for v in blk.split()], dtype=np.uint32)
        s = c.encode(vals)
        if s.size != int(nb):
            errs.append(f"fig1 block {blk}: {s.size} bytes, want {nb}")
    return errs


def sec2_prefix_sum(c) -> list[str]:
    """Sec. 2: the prefix sum of deltas (3,4,12,1) is (3,7,19,20)."""
    g = _read_golden("sec2_prefix_sum.txt")
    deltas = [int(v) for v in g["deltas"][0].split()]
    prefix = [int(v) for v in g["prefix"][0].split()]
    errs = []
    s = c.encode(np.array(prefix, dtype=np.uint32), prev=0, delta=True)
    if s.tobytes() != bytes([0] + deltas):
        errs.append(f"delta encode of {prefix}: {s.tobytes().hex()}")
    back, k = c.decode(np.array([0] + deltas, dtype=np.uint8), 4, prev=0, delta=True)
    if back.tolist() != prefix or k != 5:
        errs.append(f"delta decode of {deltas}: {back.tolist()}")
    return errs


def zero_control(c) -> list[str]:
    """Sec. 4: an all-zero control byte covers C = 4 data bytes."""
    s = np.array([0, 9, 8, 7, 6, 99, 99], dtype=np.uint8)
    back, k = c.decode(s, 4)
    if k != 5 or back.tolist() != [9, 8, 7, 6]:
        return [f"zero control byte: consumed {k}, values {back.tolist()}"]
    return []


def control_range(c) -> list[str]:
    """Sec. 4, Fig. 4: every control byte covers C in [4, 16] bytes, and
    the stream after it is consumed by exactly that many."""
    errs = []
    data = np.arange(1, 17, dtype=np.uint8)
    for cb in range(256):
        s = np.concatenate([np.array([cb], dtype=np.uint8), data])
        _, k = c.decode(s, 4)
        if not (5 <= k <= 17):
            errs.append(f"control byte {cb:#04x} consumed {k}")
    _, k0 = c.decode(np.concatenate([[0], data]).astype(np.uint8), 4)
    _, k1 = c.decode(np.concatenate([[255], data]).astype(np.uint8), 4)
    if (k0, k1) != (5, 17):
        errs.append(f"extremes 0x00/0xff consumed {k0}/{k1}")
    return errs


BOUNDARIES = [0, 1, 255, 256, 65535, 65536, (1 << 24) - 1, 1 << 24, 1 << 30, (1 << 32) - 1]


def _paper_length(x: int) -> int:
    # Sec. 3: the smallest L in {1,2,3,4} with x in [0, 2^(8L)).
    for L in (1, 2, 3, 4):
        if x < 1 << (8 * L):
            return L
    raise ValueError(x)


def length_boundaries(c) -> list[str]:
    """Sec. 3: lengths change at 2^8, 2^16 and 2^24, in every position."""
    errs = []
    for b in BOUNDARIES:
        for pos in range(4):
            vals = [7, 7, 7, 7]
            vals[pos] = b
            s = c.encode(np.array(vals, dtype=np.uint32))
            L = _paper_length(b)
            if s.size != 1 + 3 + L:
                errs.append(f"value {b} at {pos}: size {s.size}")
            if (int(s[0]) >> (2 * pos)) & 3 != L - 1:
                errs.append(f"value {b} at {pos}: control {int(s[0]):#04x}")
            back, _ = c.decode(s, 4)
            if back.tolist() != vals:
                errs.append(f"value {b} at {pos}: decodes to {back.tolist()}")
    return errs


def round_trips(c, seed: int = 11) -> list[str]:
    """decode(encode(x)) == x, plain and delta (any start, unsorted input
    wraps mod 2^32), over sizes that cover every tail n mod 4."""
    rng = np.random.default_rng(seed)
    errs = []
    for n in [0, 1, 2, 3, 4, 5, 7, 8, 13, 100, 1023, 4097]:
        for delta in (False, True):
            L = rng.integers(1, 5, n)
            x = (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (8 * (4 - L)).astype(np.uint64)).astype(np.uint32)
            prev = int(rng.integers(0, 1 << 32))
            s = c.encode(x, prev=prev, delta=delta)
            back, k = c.decode(s, n, prev=prev, delta=delta)
            if k != s.size or not np.array_equal(back, x):
                errs.append(f"round trip n={n} delta={delta}")
    return errs


def definition_agrees(c, seed: int = 12) -> list[str]:
    """Bytes and values equal those of the independent Python definition."""
    rng = np.random.default_rng(seed)
    errs = []
    for trial in range(300):
        n = int(rng.integers(0, 14))
        L = rng.integers(1, 5, n)
        x = [int(v) >> (8 * (4 - int(l))) for v, l in zip(rng.integers(0, 1 << 32, n, dtype=np.uint64), L)]
        prev = int(rng.integers(0, 1 << 32)) if trial % 2 else 0
        delta = bool(trial % 3)
        want = D.encode(x, prev, delta)
        got = c.encode(np.array(x, dtype=np.uint32), prev=prev, delta=delta).tobytes()
        if got != want:
            errs.append(f"encode {x} prev={prev} delta={delta}: {got.hex()} != {want.hex()}")
            break
    for trial in range(300):
        n = int(rng.integers(0, 14))
        raw = rng.integers(0, 256, int(rng.integers(0, 70)), dtype=np.uint8)
        prev = int(rng.integers(0, 1 << 32))
        delta = bool(trial % 2)
        wv, wk = D.decode(raw.tobytes(), n, prev, delta)
        gv, gk = c.decode(raw, n, prev=prev, delta=delta)
        if wv is None:
            if gk != (1 << 64) - 1:
                errs.append(f"random stream n={n}: truncation not reported")
                break
        elif gk != wk or gv.tolist() != wv:
            errs.append(f"random stream n={n}: {gv.tolist()} / {gk} != {wv} / {wk}")
            break
    return errs


def truncation(c) -> list[str]:
    """A stream shorter than its control bytes require is an error, and the
    decoder reads nothing beyond in_len."""
    errs = []
    x = np.array([1024, 12, 10, 1 << 30, 1, 2, 3, 1024, 5], dtype=np.uint32)
    s = c.encode(x)
    for cut in range(s.size):
        _, k = c.decode(s, x.size, in_len=cut)
        if k != (1 << 64) - 1:
            errs.append(f"in_len={cut} of {s.size}: consumed {k}")
    return errs


def pad_fields_ignored(c) -> list[str]:
    """The unused fields of an incomplete last control byte change nothing."""
    errs = []
    x = np.array([300, 5, 70000, 9, 1, 2], dtype=np.uint32)  # n mod 4 = 2
    s = c.encode(x)
    if s[1] >> 4:
        errs.append(f"encoder wrote pad fields: {int(s[1]):#04x}")
    base, k = c.decode(s, x.size)
    for pad in (0x10, 0x20, 0xF0, 0xC0):
        t = s.copy()
        t[1] |= pad
        v, k2 = c.decode(t, x.size)
        if k2 != k or not np.array_equal(v, base):
            errs.append(f"pad bits {pad:#04x} changed the result")
    return errs


def nonminimal_codes(c) -> list[str]:
    """Any code decodes, e.g. 5 stored in four bytes (Sec. 4: C is read from
    the control byte, not recomputed)."""
    s = np.array([0b11, 5, 0, 0, 0, 1, 2, 3], dtype=np.uint8)
    v, k = c.decode(s, 4)
    if k != 8 or v.tolist() != [5, 1, 2, 3]:
        return [f"non-minimal code: {v.tolist()} consumed {k}"]
    return []


def data_bytes_from_control(c) -> list[str]:
    """Sec. 4: a control byte covers C = 4 + (sum of its codes) data bytes,
    so 0x00 covers 4 and 0xFF covers 16; Fig. 3's two control bytes C1 40
    (eight integers) cover its 13 data bytes; the pad fields of an
    incomplete last control byte cover none (they code no integer).  Also,
    for random length patterns, the control bytes built here from the
    pattern cover exactly the pattern's sum of lengths."""
    errs = []
    g = _read_golden("fig3_stream.txt")
    fig3 = bytes(int(b, 16) for b in g["stream"][0].split())
    cases = [(fig3[:2], 8, 13), (b"\x00", 4, 4), (b"\xff", 4, 16),
             (b"\xff", 1, 4), (b"\xff", 2, 8), (b"\xff", 3, 12),
             (b"\xfc", 1, 1), (b"\xf0", 2, 2), (b"\xc0", 3, 3),
             (b"\xff\xff\xfc", 9, 33)]
    for ctrl, n, want in cases:
        got = c.data_bytes(np.frombuffer(ctrl, dtype=np.uint8), n)
        if got != want:
            errs.append(f"data bytes of {ctrl.hex()} for n={n}: {got}, want {want}")
    rng = np.random.default_rng(41)
    for n in (1, 2, 3, 5, 6, 7, 31, 1001):
        lens = rng.integers(1, 5, n)
        ctrl = np.zeros((n + 3) // 4, dtype=np.uint8)
        for i, L in enumerate(lens):
            ctrl[i // 4] |= np.uint8((int(L) - 1) << (2 * (i % 4)))
        if n % 4:  # pad fields set: they must still count nothing
            ctrl[-1] |= np.uint8((0xFF << (2 * (n % 4))) & 0xFF)
        got = c.data_bytes(ctrl, n)
        if got != int(lens.sum()):
            errs.append(f"data bytes of a random pattern, n={n}: {got}, want {int(lens.sum())}")
    return errs


def max_size_is_reached(c) -> list[str]:
    """The largest stream has every integer four bytes long (Sec. 3: values
    of 2^24 and above take four bytes; Sec. 4: ceil(n/4) control bytes before
    the data).  Encoding n such values, for every n mod 4, gives exactly
    svb_ref_max_compressed_size(n) bytes, and no stream of n values is longer."""
    errs = []
    rng = np.random.default_rng(42)
    for n in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 63, 1000, 4097):
        x = rng.integers(1 << 24, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        s = c.encode(x)
        if c.max_compressed_size(n) != s.size:
            errs.append(f"max size n={n}: {c.max_compressed_size(n)}, four-byte values take {s.size}")
        y = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        if c.encode(y).size > c.max_compressed_size(n):
            errs.append(f"max size n={n}: a random stream is longer")
    return errs


def _paper_query_list(rng, bits: int, n: int = 256) -> np.ndarray:
    """The setup of Sec. 5's seek/select test: n random deltas in [0, 2^b),
    prefix-summed."""
    d = rng.integers(0, 1 << bits, n, dtype=np.uint64)
    return (np.cumsum(d) & 0xFFFFFFFF).astype(np.uint32)


def seek_matches_searchsorted(c, seed: int = 31) -> list[str]:
    """Seek on sorted, differentially coded lists (Sec. 5, Fig. 6a) returns
    numpy's left insertion point and the integer there."""
    rng = np.random.default_rng(seed)
    errs = []
    for bits in (1, 4, 8, 12, 20, 24):
        x = _paper_query_list(rng, bits)
        s = c.encode(x, delta=True)
        targets = [0, int(x[0]), int(x[-1]), int(x[-1]) + 1, (1 << 32) - 1]
        targets += rng.integers(0, int(x[-1]) + 2, 40).tolist()
        for t in targets:
            t &= 0xFFFFFFFF
            want = int(np.searchsorted(x, t, side="left"))
            k, v = c.seek(s, x.size, t, delta=True)
            wv = int(x[want]) if want < x.size else 0
            if (k, v) != (want, wv):
                errs.append(f"seek b={bits} t={t}: {(k, v)} != {(want, wv)}")
    return errs


def seek_first_match_unsorted(c, seed: int = 32) -> list[str]:
    """On unsorted plain data, seek is the first position holding a value >= target."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << 20, 300).astype(np.uint32)
    s = c.encode(x)
    errs = []
    for t in rng.integers(0, 1 << 20, 50).tolist() + [0, (1 << 20) + 5]:
        hit = np.flatnonzero(x >= t)
        want = (int(hit[0]), int(x[hit[0]])) if hit.size else (x.size, 0)
        if c.seek(s, x.size, t) != want:
            errs.append(f"unsorted seek t={t}: {c.seek(s, x.size, t)} != {want}")
    return errs


def select_matches_definition(c, seed: int = 33) -> list[str]:
    """Select(i) is the i-th integer the Python definition decodes (Fig. 6b);
    i = n is out of range."""
    rng = np.random.default_rng(seed)
    errs = []
    for delta in (False, True):
        for n in (1, 5, 37):
            x = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
            prev = int(rng.integers(0, 1 << 32))
            s = c.encode(x, prev=prev, delta=delta)
            dec, _ = D.decode(s.tobytes(), n, prev, delta)
            if dec is None:
                errs.append(f"select delta={delta} n={n}: the definition rejects the stream")
                continue
            for i in range(n):
                if c.select(s, n, i, prev, delta) != dec[i]:
                    errs.append(f"select delta={delta} n={n} i={i}")
            if c.select(s, n, n, prev, delta) is not None:
                errs.append(f"select delta={delta} n={n}: index n accepted")
    return errs


def seek_select_truncation(c) -> list[str]:
    """Cutting the data stream makes exactly the answers that need the lost
    bytes fail; all control bytes are required."""
    import oracle
    x = np.array([1, 300, 70000, 5, 1 << 30, 2, 3], dtype=np.uint32)
    s = c.encode(x)
    nctrl = 2
    ends = nctrl + np.cumsum([D.length_of(int(v)) for v in x])
    errs = []
    for cut in range(s.size + 1):
        for i in range(x.size):
            got = c.select(s, x.size, i, in_len=cut)
            ok = cut >= ends[i]
            if (got is not None) != ok or (ok and got != int(x[i])):
                errs.append(f"select i={i} cut={cut}: {got}")
        k, _ = c.seek(s, x.size, 70000, in_len=cut)   # decided by index 2
        if (k != oracle.ERROR) != (cut >= ends[2]):
            errs.append(f"seek cut={cut}: {k}")
    return errs


ALL = [fig3_stream, fig1_blocks, sec2_prefix_sum, zero_control, control_range,
       length_boundaries, round_trips, definition_agrees, truncation,
       pad_fields_ignored, nonminimal_codes, data_bytes_from_control, max_size_is_reached,
       seek_matches_searchsorted,
       seek_first_match_unsorted, select_matches_definition, seek_select_truncation]


def run_all(c) -> dict[str, list[str]]:
    return {f.__name__: f(c) for f in ALL}


# --- VByte oracle pins (Sec. 2-3) -------------------------------------------

def vbyte_paper_examples(v) -> list[str]:
    """Sec. 2: 32 is one byte 00100000, 128 is 10000000 00000001."""
    g = _read_golden("vbyte_examples.txt")
    errs = []
    for line in g["example"]:
        val, hexes = line.split("=")
        val = int(val)
        want = bytes(int(b, 16) for b in hexes.split())
        got = v.encode(np.array([val], dtype=np.uint32)).tobytes()
        if got != want:
            errs.append(f"vbyte {val}: {got.hex()} != {want.hex()}")
        back, k = v.decode(np.frombuffer(want, dtype=np.uint8), 1)
        if k != len(want) or int(back[0]) != val:
            errs.append(f"vbyte decode of {want.hex()}: {back.tolist()} consumed {k}")
    return errs


def vbyte_length_boundaries(v) -> list[str]:
    """Sec. 3: lengths change at 2^7, 2^14, 2^21, 2^28 (five bytes above),
    in every position of a stream."""
    errs = []
    edges = [0, 1]
    for e in (7, 14, 21, 28):
        edges += [(1 << e) - 1, 1 << e]
    edges.append((1 << 32) - 1)
    for x in edges:
        want = D.vbyte_length(x)
        if v.length(x) != want:
            errs.append(f"vbyte length({x}) = {v.length(x)}, want {want}")
    rng = np.random.default_rng(21)
    for pos in range(4):
        for x in edges:
            vals = rng.integers(0, 128, 4).astype(np.uint32)
            vals[pos] = x
            s = v.encode(vals)
            want = sum(D.vbyte_length(int(t)) for t in vals)
            if s.size != want or v.size(vals) != want:
                errs.append(f"vbyte size with {x} at {pos}: {s.size}/{v.size(vals)}, want {want}")
    return errs


def vbyte_definition_agrees(v, seed: int = 22) -> list[str]:
    """Bytes, sizes and values equal those of the Python definition."""
    rng = np.random.default_rng(seed)
    errs = []
    for n in (1, 2, 3, 5, 17, 200):
        for delta in (False, True):
            bits = rng.integers(0, 33, n)
            x = (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (32 - bits).astype(np.uint64))
            x = x.astype(np.uint32)
            prev = int(rng.integers(0, 1 << 32))
            want = D.vbyte_encode([int(t) for t in x], prev, delta)
            got = v.encode(x, prev, delta).tobytes()
            if got != want:
                errs.append(f"vbyte n={n} delta={delta}: bytes differ")
            if v.size(x, prev, delta) != len(want):
                errs.append(f"vbyte n={n} delta={delta}: size {v.size(x, prev, delta)}")
            back, k = v.decode(np.frombuffer(want, dtype=np.uint8), n, prev, delta)
            if k != len(want) or back.tolist() != D.vbyte_decode(want, n, prev, delta) \
                    or back.tolist() != x.tolist():
                errs.append(f"vbyte n={n} delta={delta}: decode differs")
    return errs


def vbyte_truncation(v) -> list[str]:
    """A stream that ends inside an integer, or an integer over more than
    five bytes (no 32-bit value needs six), is rejected."""
    import oracle
    errs = []
    s = v.encode(np.array([1, 300, 1 << 30], dtype=np.uint32))
    for cut in range(s.size):
        _, k = v.decode(s[:cut], 3)
        if k != oracle.ERROR:
            errs.append(f"vbyte truncated at {cut}: consumed {k}")
    _, k = v.decode(np.array([0x80] * 5 + [0x01], dtype=np.uint8), 1)
    if k != oracle.ERROR:
        errs.append("vbyte six-byte integer accepted")
    return errs


def run_all_vbyte(v) -> dict[str, list[str]]:
    return {f.__name__: f(v) for f in (vbyte_paper_examples, vbyte_length_boundaries,
                                       vbyte_definition_agrees, vbyte_truncation)}
