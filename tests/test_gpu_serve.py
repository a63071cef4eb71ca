"""The serving loop: every request's result is the same whether it is served
alone or in a mix of concurrent, batched requests, and equals the oracle's."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    from paper_1709_08990_gb300.batch import ListPool
    L = W.lists_lengths(400, cap=4_000_000)
    vals, first = W.posting_lists(4, L)
    p = ListPool(L, vals, delta=True)
    p.h_vals, p.h_first = vals, first
    return p


def _serve(pool, req, **kw):
    from paper_1709_08990_gb300.serve import Collector, Server
    srv = Server(pool, **kw)
    col = Collector()
    out = srv.run(req, collect=col)
    assert np.all(np.isfinite(out["done"]))
    return col.results, out


def test_results_same_alone_and_in_the_mix(pool):
    req = W.serve_requests(pool.lengths, 300, None, seed=5, encode_fraction=0.2)
    mix, out_mix = _serve(pool, req, budget=64 << 20, max_batch=4096, slots=2)
    assert out_mix["batches"] < 300           # requests were really batched together
    alone, out_alone = _serve(pool, req, budget=64 << 20, max_batch=1, slots=1)
    assert out_alone["batches"] == 300
    for i in range(300):
        assert np.array_equal(mix[i], alone[i]), f"request {i}"
        if req.is_encode[i]:
            f = int(req.enc_first[i])
            want = oracle.encode(req.enc_values[f:f + int(req.n[i])], delta=True)
        else:
            j = int(req.list_id[i])
            want = pool.h_vals[int(pool.h_first[j]):int(pool.h_first[j]) + int(pool.lengths[j])]
        assert np.array_equal(mix[i], want), f"request {i} differs from the oracle"


def test_small_budget_admits_in_waves(pool):
    """A scratch budget far below the mix's total: requests wait for earlier
    batches to free their blocks, and still come out right."""
    req = W.serve_requests(pool.lengths, 200, None, seed=6, encode_fraction=0.1)
    need = int((4 * req.n).sum())
    budget = max(1 << 20, need // 8)
    res, out = _serve(pool, req, budget=budget, max_batch=4096, slots=2)
    assert out["batches"] >= 4
    for i in range(200):
        if not req.is_encode[i]:
            j = int(req.list_id[i])
            want = pool.h_vals[int(pool.h_first[j]):int(pool.h_first[j]) + int(pool.lengths[j])]
            assert np.array_equal(res[i], want)


def test_open_loop_arrivals(pool):
    """Poisson arrivals: every request completes after it arrived."""
    req = W.serve_requests(pool.lengths, 500, 20000.0, seed=7)
    from paper_1709_08990_gb300.serve import Server, summarize
    srv = Server(pool, budget=64 << 20)
    out = srv.run(req)
    assert np.all(out["done"] >= req.arrival)
    s = summarize(req, out)
    assert s["p99_ms"] >= s["p50_ms"] > 0


@pytest.mark.parametrize("tile", [4096, 8192])
def test_host_plan_matches_the_library_layout(tile):
    """serve.host_plan writes the plan layout the batched kernels read: its
    header and big-list order equal the library's plan for the same lists
    (no units), at either decode tile."""
    from paper_1709_08990_gb300 import svb
    from paper_1709_08990_gb300.serve import PLAN_HEADER_WORDS, host_plan
    n = np.array([5, 70_000, 9000, 8192, 3, 20_000, 20_000, 100, 8191], dtype=np.uint32)
    lists = np.zeros(n.size, dtype=svb.list_dtype())
    lists["n"] = n
    nb = svb.svb_batch_plan_bytes(n.size)
    d = torch.zeros(nb, dtype=torch.uint8, device="cuda:0")
    try:
        assert svb.svb_batch_set_tile(tile) == 0
        assert svb.svb_batch_plan_segments(lists, n.size, 8192, 0, d, nb) == 0
        lib = d.cpu().numpy().view(np.uint32)
        host = host_plan(n, 8192, tile_quads=svb.svb_batch_get_tile() // 4)
    finally:
        svb.svb_batch_set_tile(0)
    h = PLAN_HEADER_WORDS
    assert np.array_equal(lib[:h], host[:h])
    nbig = int(host[0])
    assert np.array_equal(lib[h:h + nbig], host[h:h + nbig])
    assert sorted(lib[h + nbig:h + n.size].tolist()) == sorted(host[h + nbig:].tolist())
