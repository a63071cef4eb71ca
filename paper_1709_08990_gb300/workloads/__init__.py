"""Seeded synthetic workloads (counter-based SplitMix64; see ``gen.c``).

Random numbers and value distributions only: this module computes nothing
of the codec.  The tests of both the CUDA path and the oracle draw their
inputs here, so both sides always see the same integers.

The five workloads mirror the paper's posting-list setting (Sec. 5: sorted
document ids, differential coding, lists grouped by length, longer lists
more compressible) with synthetic data, because the ClueWeb09 lists the
paper measured are not available:

  uniform_1m    n = 2^20, byte length ~ U{1..4}, value uniform in its length's
                range, seed 1 (unpredictable control pattern)
  delta_64m     n = 2^26 sorted, gaps geometric with mean 16 on {1, 2, ...},
                start 0, seed 2
  skewed_1g     n = 2^30, P(length) = (.50, .30, .15, .05), seed 3
  lists_100k    100,000 sorted lists, lengths log-uniform on [8, 4194304]
                scaled to a total of at most 2^30, ids < 2^31 with geometric
                gaps of mean 2^31/(m+1), seed 4
  serve         the lists_100k pool plus fresh lists drawn with seed 5
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsvbgen.so")


def build_cmd() -> list[str]:
    return ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", _LIB, _SRC,
            "-lm", "-lpthread"]


def build() -> None:
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return
    subprocess.run(build_cmd(), check=True)


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, sz, vp, i32 = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int
        L.svbgen_word.argtypes = [u64, ctypes.c_uint32, u64]
        L.svbgen_word.restype = u64
        for f in (L.svbgen_uniform_lengths, L.svbgen_skewed_lengths):
            f.argtypes = [u64, sz, vp, i32]
            f.restype = None
        L.svbgen_sorted_geometric.argtypes = [u64, sz, ctypes.c_double, ctypes.c_uint32, vp, i32]
        L.svbgen_sorted_geometric.restype = None
        L.svbgen_list_lengths.argtypes = [u64, sz, ctypes.c_uint32, ctypes.c_uint32, u64, vp]
        L.svbgen_list_lengths.restype = u64
        L.svbgen_posting_lists.argtypes = [u64, sz, vp, vp, vp, i32]
        L.svbgen_posting_lists.restype = None
        L.svbgen_posting_list.argtypes = [u64, u64, ctypes.c_uint32, vp]
        L.svbgen_posting_list.restype = ctypes.c_int
        _lib = L
    return _lib


def _out(n: int, out: np.ndarray | None) -> np.ndarray:
    if out is None:
        return np.empty(n, dtype=np.uint32)
    assert out.dtype == np.uint32 and out.size >= n and out.flags.c_contiguous
    return out


def word(seed: int, stream: int, i: int) -> int:
    return lib().svbgen_word(seed, stream, i)


def uniform_lengths(seed: int, n: int, out=None, threads: int = 0) -> np.ndarray:
    a = _out(n, out)
    lib().svbgen_uniform_lengths(seed, n, a.ctypes.data, threads)
    return a[:n]


def skewed_lengths(seed: int, n: int, out=None, threads: int = 0) -> np.ndarray:
    a = _out(n, out)
    lib().svbgen_skewed_lengths(seed, n, a.ctypes.data, threads)
    return a[:n]


def sorted_geometric(seed: int, n: int, mean: float = 16.0, start: int = 0,
                     out=None, threads: int = 0) -> np.ndarray:
    a = _out(n, out)
    lib().svbgen_sorted_geometric(seed, n, float(mean), start, a.ctypes.data, threads)
    return a[:n]


def list_lengths(seed: int, k: int, lo: int = 8, hi: int = 4194304,
                 cap: int = 1 << 30) -> np.ndarray:
    a = np.empty(k, dtype=np.uint32)
    lib().svbgen_list_lengths(seed, k, lo, hi, cap, a.ctypes.data)
    return a


def posting_lists(seed: int, lengths: np.ndarray, out=None, threads: int = 0):
    """(ids of all lists back to back, first index of each list)."""
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    first = np.zeros(lengths.size, dtype=np.uint64)
    if lengths.size > 1:
        first[1:] = np.cumsum(lengths[:-1], dtype=np.uint64)
    total = int(lengths.sum(dtype=np.uint64))
    a = _out(total, out)
    lib().svbgen_posting_lists(seed, lengths.size, lengths.ctypes.data,
                               first.ctypes.data, a.ctypes.data, threads)
    return a[:total], first


def posting_list(seed: int, first: int, m: int) -> np.ndarray:
    a = np.empty(max(1, m), dtype=np.uint32)
    lib().svbgen_posting_list(seed, first, m, a.ctypes.data)
    return a[:m]


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "array" or "lists"
    n: int             # integers (total over lists for "lists")
    delta: bool
    seed: int
    description: str


WORKLOADS = {
    "uniform_1m": Workload("uniform_1m", "array", 1 << 20, False, 1,
                           "plain encode+decode, n=2^20, length ~ U{1..4}"),
    "delta_64m": Workload("delta_64m", "array", 1 << 26, True, 2,
                          "delta encode+decode, n=2^26 sorted, geometric gaps mean 16, start 0"),
    "skewed_1g": Workload("skewed_1g", "array", 1 << 30, False, 3,
                          "plain decode, n=2^30, P(length)=(.50,.30,.15,.05)"),
    "lists_100k": Workload("lists_100k", "lists", 1 << 30, True, 4,
                           "100,000 sorted lists, log-uniform lengths [8, 4194304] "
                           "capped at 2^30 total, geometric gaps mean 2^31/(m+1)"),
}


def array_values(name: str, n: int | None = None, out=None, threads: int = 0) -> np.ndarray:
    """Values of a single-array workload; n < full size gives its prefix."""
    w = WORKLOADS[name]
    n = w.n if n is None else n
    if name == "uniform_1m":
        return uniform_lengths(w.seed, n, out, threads)
    if name == "delta_64m":
        return sorted_geometric(w.seed, n, 16.0, 0, out, threads)
    if name == "skewed_1g":
        return skewed_lengths(w.seed, n, out, threads)
    raise KeyError(name)


def lists_lengths(num_lists: int = 100_000, cap: int = 1 << 30) -> np.ndarray:
    return list_lengths(WORKLOADS["lists_100k"].seed, num_lists, 8, 4194304, cap)


# ---------------------------------------------------------------------------
# Serving workload: requests over a pool of lists (seeded, reproducible).

@dataclass
class RequestStream:
    arrival: np.ndarray      # seconds from the start, non-decreasing
    is_encode: np.ndarray    # bool
    list_id: np.ndarray      # decode: pool list id; encode: -1
    n: np.ndarray            # integers of the request
    enc_first: np.ndarray    # encode: index of the fresh list in enc_values; else -1
    enc_values: np.ndarray   # fresh lists for the encode requests, back to back


def zipf_ranks(rng, count: int, num_ranks: int, s: float = 1.1) -> np.ndarray:
    """Ranks 0..num_ranks-1 drawn with P(rank r) proportional to (r+1)^-s."""
    w = np.arange(1, num_ranks + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return np.minimum(np.searchsorted(cdf, rng.random(count), side="right"), num_ranks - 1)


def serve_requests(pool_lengths: np.ndarray, count: int, rate: float | None,
                   seed: int = 5, encode_fraction: float = 0.05, s: float = 1.1,
                   fresh_threads: int = 0) -> RequestStream:
    """count requests over a pool of lists.  rate = mean arrivals per second
    (Poisson; None puts every arrival at time 0).  Decode requests pick a
    list by Zipf(s) over popularity ranks mapped to list ids by a seeded
    permutation; encode requests carry a fresh sorted list whose length is
    that of a uniformly drawn pool list, drawn like the pool's lists."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = pool_lengths.size
    perm = rng.permutation(k)
    if rate is None:
        arrival = np.zeros(count)
    else:
        arrival = np.cumsum(rng.exponential(1.0 / rate, count))
    is_enc = rng.random(count) < encode_fraction
    list_id = perm[zipf_ranks(rng, count, k, s)]
    n = pool_lengths[list_id].astype(np.int64)
    enc_len = pool_lengths[rng.integers(0, k, count)].astype(np.int64)
    n = np.where(is_enc, enc_len, n)
    list_id = np.where(is_enc, -1, list_id)
    enc_idx = np.flatnonzero(is_enc)
    enc_first = np.full(count, -1, dtype=np.int64)
    lens = n[enc_idx].astype(np.uint32)
    if enc_idx.size:
        firsts = np.zeros(enc_idx.size, dtype=np.int64)
        firsts[1:] = np.cumsum(lens[:-1], dtype=np.int64)
        enc_first[enc_idx] = firsts
        # A fresh stream of the list generator (seed of this workload).
        vals, _ = posting_lists(seed, lens, threads=fresh_threads)
    else:
        vals = np.zeros(0, dtype=np.uint32)
    return RequestStream(arrival, is_enc, list_id, n, enc_first, vals)
