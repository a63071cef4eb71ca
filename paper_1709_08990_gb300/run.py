"""Run one codec operation repeatedly on a synthetic workload and print the
mean time per call (CUDA events on the launching stream).

    python -m paper_1709_08990_gb300.run OP [--workload W] [--n N] [--reps R]

OP is one of
  decode        svb_decode_async on a single-array workload (differential
                when the workload is)
  encode        svb_encode_async on a single-array workload
  batch_decode  svb_batch_decode of the list workload (one persistent launch)
  batch_encode  svb_batch_encode of the list workload
  size          svb_size_report_async on a single-array workload
  query         svb_query_batch: seeks on --lists lists of 256 integers
                (deltas below 2^--bits), --n queries
  append        svb_append of 2^20 integers to a --n integer array

The input is generated and, for decoding, encoded before the timed calls; the
first call's result is checked against the generated values.  Meant for
timing one kernel in isolation and as the command under a profiler.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import svb
from . import workloads as W


def _time(fn, reps: int, stream) -> float:
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _array(op: str, name: str, n: int, reps: int) -> dict:
    w = W.WORKLOADS[name]
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(W.array_values(name, n=n).view(np.int32)).to(dev)
    stream = torch.cuda.current_stream()
    ws_bytes = svb.svb_workspace_size(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    svb.svb_workspace_init(ws, ws_bytes, stream)
    stream_bytes = svb.encode(x, delta=w.delta)
    if op == "encode":
        out = torch.empty(svb.svb_max_compressed_size(n), dtype=torch.uint8, device=dev)

        def fn():
            st = svb.svb_encode_async(x, n, out, 0, int(w.delta), res, ws, ws_bytes, stream)
            if st != 0:
                raise svb.SvbError(st, "svb_encode_async")

        ms = _time(fn, reps, stream)
        k = stream_bytes.numel()
        ok = int(res[0].item()) == k and bool(torch.equal(out[:k], stream_bytes))
    else:
        out = torch.empty(n, dtype=torch.int32, device=dev)
        k = stream_bytes.numel()

        def fn():
            st = svb.svb_decode_async(stream_bytes, k, n, out, 0, int(w.delta), res, ws,
                                      ws_bytes, stream)
            if st != 0:
                raise svb.SvbError(st, "svb_decode_async")

        ms = _time(fn, reps, stream)
        ok = int(res[0].item()) == k and bool(torch.equal(out, x))
    return {"op": op, "workload": name, "n": n, "delta": w.delta,
            "stream_bytes": int(stream_bytes.numel()), "ms": ms,
            "gints_per_s": n / (ms / 1e3) / 1e9, "verified": ok}


def _lists(op: str, name: str, count: int, reps: int, cap: int = 1 << 30,
           segment_tiles: int | None = None) -> dict:
    from .batch import ListPool
    dev = torch.device("cuda", torch.cuda.current_device())
    lengths = W.lists_lengths(count, cap)
    total = int(lengths.sum(dtype=np.uint64))
    vals = np.empty(total, dtype=np.uint32)
    W.posting_lists(W.WORKLOADS[name].seed, lengths, out=vals)
    d_vals = torch.from_numpy(vals.view(np.int32)).to(dev)
    pool = ListPool(lengths, d_vals, delta=True, device=dev, segment_tiles=segment_tiles)
    stream = torch.cuda.current_stream()
    if op == "batch_decode":
        out = torch.empty(total, dtype=torch.int32, device=dev)
        ms = _time(lambda: pool.decode(out), reps, stream)
        ok = bool(torch.equal(out, d_vals))
    else:
        out = torch.empty_like(pool.pool)
        ms = _time(lambda: pool.encode(out), reps, stream)
        ok = bool(torch.equal(out, pool.pool))
    return {"op": op, "workload": name, "lists": count, "n": total,
            "tile_ints": svb.svb_batch_get_tile(),
            "stages": svb.svb_batch_get_stages(int(op == "batch_encode")),
            "stream_bytes": pool.pool_bytes, "ms": ms,
            "gints_per_s": total / (ms / 1e3) / 1e9, "verified": ok}


def _size(name: str, n: int, reps: int) -> dict:
    w = W.WORKLOADS[name]
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(W.array_values(name, n=n).view(np.int32)).to(dev)
    stream = torch.cuda.current_stream()
    d = torch.zeros(2, dtype=torch.int64, device=dev)

    def fn():
        st = svb.svb_size_report_async(x, n, 0, int(w.delta), d, stream)
        if st != 0:
            raise svb.SvbError(st, "svb_size_report_async")

    ms = _time(fn, reps, stream)
    k = svb.encode(x, delta=w.delta).numel()
    return {"op": "size", "workload": name, "n": n, "ms": ms,
            "gints_per_s": n / (ms / 1e3) / 1e9, "verified": int(d[0].item()) == k}


def _query(num_lists: int, nq: int, bits: int, reps: int) -> dict:
    from .batch import ListPool
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(600 + bits)
    d = rng.integers(0, 1 << bits, (num_lists, 256), dtype=np.uint64)
    vals = (np.cumsum(d, axis=1) & 0xFFFFFFFF).astype(np.uint32)
    pool = ListPool(np.full(num_lists, 256, dtype=np.uint32), vals.reshape(-1), delta=True,
                    device=dev)
    d_tab = torch.from_numpy(pool.dec_table.view(np.uint8).copy()).to(dev)
    q = np.zeros(nq, dtype=svb.query_dtype())
    q["list"] = rng.integers(0, num_lists, nq)
    q["op"] = svb.SVB_SEEK
    q["arg"] = (rng.random(nq) * (vals[q["list"], -1].astype(np.uint64) + 1)).astype(np.uint64)
    d_q = torch.from_numpy(q.view(np.uint8).copy()).to(dev)
    d_a = torch.zeros(nq * svb.answer_dtype().itemsize, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ms = _time(lambda: svb.svb_query_batch(d_tab, num_lists, pool.pool, 1, d_q, nq, d_a, stream),
               reps, stream)
    a = d_a.cpu().numpy().view(svb.answer_dtype())
    k = rng.integers(0, nq, 64)
    ok = all(int(a["index"][i]) == int(np.searchsorted(vals[int(q["list"][i])], int(q["arg"][i])))
             for i in k)
    return {"op": "query", "lists": num_lists, "queries": nq, "bits": bits, "ms": ms,
            "mqueries_per_s": nq / ms / 1e3, "verified": bool(ok)}


def _append(n0: int, k: int, reps: int) -> dict:
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(W.array_values("skewed_1g", n=n0 + k).view(np.int32)).to(dev)
    s = svb.encode(x[:n0])
    nc = (n0 + 3) // 4
    ctrl_cap, data_cap = (n0 + k + 3) // 4 + 8, s.numel() - nc + 4 * k + 64
    d_ctrl = torch.zeros(ctrl_cap, dtype=torch.uint8, device=dev)
    d_data = torch.zeros(data_cap, dtype=torch.uint8, device=dev)
    c0, dat0, dl0 = s[:nc].clone(), s[nc:].clone(), s.numel() - nc
    t = 0.0
    for i in range(reps + 1):
        d_ctrl[:nc].copy_(c0)
        d_data[:dl0].copy_(dat0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dl = svb.svb_append(d_ctrl, ctrl_cap, d_data, data_cap, dl0, n0, x[n0:], k, 0, 0)
        if i:
            t += time.perf_counter() - t0
    whole = svb.encode(x)
    nc1 = (n0 + k + 3) // 4
    ok = bool(torch.equal(d_ctrl[:nc1], whole[:nc1])) and bool(torch.equal(d_data[:dl], whole[nc1:]))
    ms = t / max(1, reps) * 1e3
    return {"op": "append", "n0": n0, "k": k, "ms": ms, "gints_per_s": k / ms / 1e6,
            "verified": ok}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_1709_08990_gb300.run")
    ap.add_argument("op", choices=["decode", "encode", "batch_decode", "batch_encode", "size",
                                   "query", "append"])
    ap.add_argument("--workload", default=None)
    ap.add_argument("--n", type=int, default=0, help="integers (array workloads; 0 = full)")
    ap.add_argument("--lists", type=int, default=100_000, help="lists (list workload)")
    ap.add_argument("--cap", type=int, default=1 << 30,
                    help="total integers the list lengths are scaled to (list workload); "
                         "--lists 12500 --cap 134217728 is lists_100k at 1/8 scale")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--bits", type=int, default=8, help="query: deltas below 2^bits")
    ap.add_argument("--segment-tiles", type=int, default=-1,
                    help="batch: tiles per unit of a split list (0: no splitting; "
                         "-1: the library's default)")
    ap.add_argument("--tile", type=int, default=0,
                    help="batch_decode: decode tile, 4096 or 8192 integers (0: the default)")
    ap.add_argument("--stages", type=int, default=0,
                    help="batch: staging depth of the batched kernel (0: the default)")
    ap.add_argument("--variant", type=int, default=0,
                    help="decoder variant (svb_set_decode_variant), 0 = the default")
    ap.add_argument("--kernels", action="store_true",
                    help="also time each library kernel (CUDA events around every launch)")
    a = ap.parse_args(argv)
    if svb.svb_set_decode_variant(a.variant) != 0:
        raise SystemExit(f"unknown decoder variant {a.variant}")
    if a.kernels:
        svb.svb_profile_begin()
    if a.op.startswith("batch"):
        enc = a.op == "batch_encode"
        if (svb.svb_batch_set_tile(a.tile) != 0 or
                svb.svb_batch_set_stages(0 if enc else a.stages, a.stages if enc else 0) != 0):
            raise SystemExit(f"tile {a.tile} / staging depth {a.stages} not built")
        r = _lists(a.op, a.workload or "lists_100k", a.lists, a.reps, a.cap,
                   None if a.segment_tiles < 0 else a.segment_tiles)
    elif a.op == "size":
        name = a.workload or "skewed_1g"
        r = _size(name, a.n or W.WORKLOADS[name].n, a.reps)
    elif a.op == "query":
        r = _query(a.lists, a.n or (1 << 20), a.bits, a.reps)
    elif a.op == "append":
        r = _append(a.n or (1 << 24), 1 << 20, a.reps)
    else:
        name = a.workload or "skewed_1g"
        r = _array(a.op, name, a.n or W.WORKLOADS[name].n, a.reps)
    if a.kernels:
        torch.cuda.synchronize()
        r["kernels_ms"] = {k: t / c for k, (c, t) in svb.profile_end().items()}
    r["variant"] = a.variant
    print(json.dumps(r), flush=True)
    if not r["verified"]:
        raise SystemExit("result differs from the generated values")


if __name__ == "__main__":
    main()
