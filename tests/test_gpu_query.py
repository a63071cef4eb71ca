"""GPU seek/select on compressed lists (Sec. 5, Fig. 6) against the oracle,
query by query."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import svb
from paper_1709_08990_gb300.batch import ListPool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def paper_lists(rng, count: int, bits: int, lengths=None) -> tuple[np.ndarray, np.ndarray]:
    """Lists built as in Sec. 5's seek/select test: random deltas in [0, 2^b),
    prefix-summed (256 integers each unless lengths say otherwise)."""
    if lengths is None:
        lengths = np.full(count, 256, dtype=np.uint32)
    parts = []
    for m in lengths:
        d = rng.integers(0, 1 << bits, int(m), dtype=np.uint64)
        parts.append((np.cumsum(d) & 0xFFFFFFFF).astype(np.uint32))
    return lengths.astype(np.uint32), np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def run_queries(pool: ListPool, table: np.ndarray, queries: np.ndarray, delta: bool) -> np.ndarray:
    d_tab = torch.from_numpy(table.view(np.uint8).copy()).to(DEV)
    d_q = torch.from_numpy(queries.view(np.uint8).copy()).to(DEV)
    d_a = torch.zeros(queries.size * svb.answer_dtype().itemsize, dtype=torch.uint8, device=DEV)
    st = svb.svb_query_batch(d_tab, table.size, pool.pool, int(delta), d_q, queries.size, d_a)
    assert st == 0
    torch.cuda.synchronize()
    return d_a.cpu().numpy().view(svb.answer_dtype())


def oracle_answer(host_pool, entry, q, delta) -> tuple[int, int, int]:
    c = oracle.codec()
    s = host_pool[int(entry["in_off"]): int(entry["in_off"]) + int(entry["in_len"])]
    n = int(entry["n"])
    if q["op"] == svb.SVB_SEEK:
        k, v = c.seek(s, n, int(q["arg"]), int(entry["prev"]), delta)
        if k == oracle.ERROR:
            return None, 0, svb.SVB_ETRUNCATED
        return k, v, 0
    v = c.select(s, n, int(q["arg"]), int(entry["prev"]), delta)
    if int(q["arg"]) >= n:
        return int(q["arg"]), 0, svb.SVB_EINVAL
    if v is None:
        return int(q["arg"]), 0, svb.SVB_ETRUNCATED
    return int(q["arg"]), v, 0


def make_queries(rng, lengths, values, firsts, count):
    q = np.zeros(count, dtype=svb.query_dtype())
    q["list"] = rng.integers(0, lengths.size, count)
    q["op"] = rng.integers(0, 2, count)
    for k in range(count):
        li = int(q["list"][k])
        m = int(lengths[li])
        seg = values[int(firsts[li]): int(firsts[li]) + m]
        if q["op"][k] == svb.SVB_SEEK:
            choice = rng.integers(0, 6)
            hi = int(seg.max()) if m else 0
            q["arg"][k] = [0, int(seg[0]) if m else 0, hi, min(hi + 1, (1 << 32) - 1),
                           int(rng.integers(0, hi + 2)), int(rng.integers(0, hi + 2))][choice]
        else:
            q["arg"][k] = int(rng.integers(0, max(1, m)))
    return q


def check(pool, table, queries, delta):
    got = run_queries(pool, table, queries, delta)
    host_pool = pool.pool.cpu().numpy()
    for k in range(queries.size):
        q = queries[k]
        idx, val, st = oracle_answer(host_pool, table[int(q["list"])], q, delta)
        a = got[k]
        assert int(a["status"]) == st, (k, q, a)
        if st == 0:
            assert (int(a["index"]), int(a["value"])) == (idx, val), (k, q, a)


@pytest.mark.parametrize("bits", [1, 8, 12, 24])
def test_paper_lists_seek_select(bits):
    rng = np.random.default_rng(100 + bits)
    lengths, values = paper_lists(rng, 300, bits)
    pool = ListPool(lengths, values, delta=True, device=DEV)
    firsts = np.concatenate([[0], np.cumsum(lengths[:-1], dtype=np.uint64)])
    q = make_queries(rng, lengths, values, firsts, 1500)
    check(pool, pool.dec_table, q, True)


@pytest.mark.parametrize("delta", [False, True])
def test_ragged_lengths(delta):
    rng = np.random.default_rng(7)
    lengths = np.array([1, 2, 3, 4, 5, 127, 128, 129, 130, 511, 512, 513, 1000, 4097, 9],
                       dtype=np.uint32)
    if delta:
        _, values = paper_lists(rng, lengths.size, 16, lengths)
    else:
        values = rng.integers(0, 1 << 32, int(lengths.sum()), dtype=np.uint64).astype(np.uint32)
    pool = ListPool(lengths, values, delta=delta, device=DEV)
    firsts = np.concatenate([[0], np.cumsum(lengths[:-1], dtype=np.uint64)])
    q = make_queries(rng, lengths, values, firsts, 2000)
    check(pool, pool.dec_table, q, delta)


def test_truncated_lists_and_invalid_queries():
    rng = np.random.default_rng(8)
    lengths, values = paper_lists(rng, 40, 20, np.full(40, 300, dtype=np.uint32))
    pool = ListPool(lengths, values, delta=True, device=DEV)
    table = pool.dec_table.copy()
    nq = (table["n"].astype(np.int64) + 3) // 4
    # cut some lists inside their data, one inside its control bytes
    for li in range(0, 40, 3):
        table["in_len"][li] = nq[li] + rng.integers(0, int(table["in_len"][li] - nq[li]))
    table["in_len"][1] = nq[1] - 1
    firsts = np.concatenate([[0], np.cumsum(lengths[:-1], dtype=np.uint64)])
    q = make_queries(rng, lengths, values, firsts, 1500)
    check(pool, table, q, True)
    bad = np.zeros(3, dtype=svb.query_dtype())
    bad[0] = (40, svb.SVB_SEEK, 5)       # no such list
    bad[1] = (0, svb.SVB_SELECT, 300)    # index == n
    bad[2] = (0, 7, 0)                   # unknown op
    got = run_queries(pool, table, bad, True)
    assert got["status"].tolist() == [svb.SVB_EINVAL] * 3
