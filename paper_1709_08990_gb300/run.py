"""Run one codec operation repeatedly on a synthetic workload and print the
mean time per call (CUDA events on the launching stream).

    python -m paper_1709_08990_gb300.run OP [--workload W] [--n N] [--reps R]

OP is one of
  decode        svb_decode_async on a single-array workload (differential
                when the workload is)
  encode        svb_encode_async on a single-array workload
  batch_decode  svb_batch_decode of the list workload (one persistent launch)
  batch_encode  svb_batch_encode of the list workload

The input is generated and, for decoding, encoded before the timed calls; the
first call's result is checked against the generated values.  Meant for
timing one kernel in isolation and as the command under a profiler.
"""
from __future__ import annotations

import argparse
import json

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


def _lists(op: str, name: str, count: int, reps: int, cap: int = 1 << 30) -> dict:
    from .batch import ListPool
    dev = torch.device("cuda", torch.cuda.current_device())
    lengths = W.lists_lengths(count, cap)
    total = int(lengths.sum(dtype=np.uint64))
    vals = np.empty(total, dtype=np.uint32)
    W.posting_lists(W.WORKLOADS[name].seed, lengths, out=vals)
    d_vals = torch.from_numpy(vals.view(np.int32)).to(dev)
    pool = ListPool(lengths, d_vals, delta=True, device=dev)
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
            "stream_bytes": pool.pool_bytes, "ms": ms,
            "gints_per_s": total / (ms / 1e3) / 1e9, "verified": ok}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_1709_08990_gb300.run")
    ap.add_argument("op", choices=["decode", "encode", "batch_decode", "batch_encode"])
    ap.add_argument("--workload", default=None)
    ap.add_argument("--n", type=int, default=0, help="integers (array workloads; 0 = full)")
    ap.add_argument("--lists", type=int, default=100_000, help="lists (list workload)")
    ap.add_argument("--cap", type=int, default=1 << 30,
                    help="total integers the list lengths are scaled to (list workload); "
                         "--lists 12500 --cap 134217728 is lists_100k at 1/8 scale")
    ap.add_argument("--reps", type=int, default=10)
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
        r = _lists(a.op, a.workload or "lists_100k", a.lists, a.reps, a.cap)
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
