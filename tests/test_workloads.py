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


def test_serve_requests_follow_the_recipe():
    """Poisson arrivals, 5 % encodes of fresh sorted lists, decodes of pool
    lists chosen Zipf(1.1) over ranks mapped to ids by a permutation."""
    k = 2000
    pool = W.list_lengths(11, k, 8, 5000)
    count, rate = 20000, 1e5
    r = W.serve_requests(pool, count, rate, seed=5)
    assert np.all(np.diff(r.arrival) >= 0)
    gaps = np.diff(np.concatenate([[0.0], r.arrival]))
    assert abs(gaps.mean() * rate - 1) < 0.05          # mean 1/rate
    assert abs(np.std(gaps) * rate - 1) < 0.05         # exponential: sd = mean
    frac = r.is_encode.mean()
    assert abs(frac - 0.05) < 0.01
    dec = ~r.is_encode
    assert np.all((r.list_id[dec] >= 0) & (r.list_id[dec] < k))
    assert np.array_equal(r.n[dec], pool[r.list_id[dec]])
    assert np.all(r.list_id[r.is_encode] == -1) and np.all(r.enc_first[dec] == -1)
    # Zipf(1.1): the most requested list takes 1 / H_{k,1.1} of the decodes
    counts = np.bincount(r.list_id[dec], minlength=k)
    h = np.sum(np.arange(1, k + 1, dtype=np.float64) ** -1.1)
    assert abs(counts.max() / dec.sum() - 1 / h) < 0.02
    top, second = np.sort(counts)[-1], np.sort(counts)[-2]
    assert 1.8 < top / second < 2.6                    # rank 1 / rank 2 = 2^1.1 = 2.14
    # fresh lists: back to back, each strictly increasing below 2^31
    e = np.flatnonzero(r.is_encode)
    ends = r.enc_first[e] + r.n[e]
    assert r.enc_first[e[0]] == 0 and np.array_equal(r.enc_first[e[1:]], ends[:-1])
    assert r.enc_values.size == ends[-1]
    for j in e[:50]:
        v = r.enc_values[r.enc_first[j]:r.enc_first[j] + r.n[j]].astype(np.int64)
        assert np.all(np.diff(v) > 0) and v[-1] < (1 << 31)


def test_serve_requests_are_reproducible_and_burst_at_time_zero():
    pool = W.list_lengths(12, 100, 8, 1000)
    a = W.serve_requests(pool, 500, None, seed=7)
    b = W.serve_requests(pool, 500, None, seed=7)
    assert np.all(a.arrival == 0)
    for f in ("is_encode", "list_id", "n", "enc_first", "enc_values"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = W.serve_requests(pool, 500, None, seed=8)
    assert not np.array_equal(a.list_id, c.list_id)
