"""The seeded workload generators (no GPU needed)."""
from __future__ import annotations

import numpy as np

from paper_1709_08990_gb300 import workloads as W


def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    # 0x06c45d188009454f (Steele, Lea, Flood 2014); state k*gamma gives the
    # (k+1)-th output.
    g = 0x9E3779B97F4A7C15
    assert W.word(0, 0, 0) == 0xE220A8397B1DCDAF
    assert W.word(0, 0, g) == 0x6E789E6AA1B965F4
    assert W.word(0, 0, (2 * g) % (1 << 64)) == 0x06C45D188009454F


def test_thread_count_does_not_change_values():
    for f in (W.uniform_lengths, W.skewed_lengths):
        a = f(7, 300_001, threads=1)
        b = f(7, 300_001, threads=5)
        assert np.array_equal(a, b)
    a = W.sorted_geometric(3, 200_000, 16.0, 5, threads=1)
    b = W.sorted_geometric(3, 200_000, 16.0, 5, threads=7)
    assert np.array_equal(a, b)


def _lengths(x):
    return np.where(x < 1 << 8, 1, np.where(x < 1 << 16, 2, np.where(x < 1 << 24, 3, 4)))


def test_uniform_and_skewed_length_mix():
    h = np.bincount(_lengths(W.array_values("uniform_1m")), minlength=5)[1:] / (1 << 20)
    assert np.allclose(h, 0.25, atol=0.005)
    h = np.bincount(_lengths(W.array_values("skewed_1g", n=1 << 22)), minlength=5)[1:] / (1 << 22)
    assert np.allclose(h, [0.50, 0.30, 0.15, 0.05], atol=0.005)


def test_sorted_geometric():
    x = W.array_values("delta_64m", n=1 << 22)
    g = np.diff(np.concatenate([[0], x.astype(np.int64)]))
    assert g.min() >= 1
    assert abs(g.mean() - 16.0) < 0.05


def test_list_lengths_and_lists():
    L = W.lists_lengths()
    assert L.size == 100_000 and L.min() >= 8 and int(L.sum()) <= 1 << 30
    assert int(L.sum()) > (1 << 30) - 100_000 * 8
    assert (L % 4 != 0).sum() > 50_000
    sub = L[:500]
    v, first = W.posting_lists(4, sub)
    assert v.size == int(sub.sum())
    for j in range(0, 500, 37):
        lst = v[int(first[j]):int(first[j]) + int(sub[j])].astype(np.int64)
        assert np.all(np.diff(lst) > 0) and lst.max() < 1 << 31 and lst.min() >= 1
    one = W.posting_list(4, int(first[37]), int(sub[37]))
    assert np.array_equal(one, v[int(first[37]):int(first[37]) + int(sub[37])])
