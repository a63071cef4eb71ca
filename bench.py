"""Stream VByte decode throughput on GB300.

One step = one decode of the whole workload array (control-length reduce,
look-back offset scan, staging, gather, stores: the decode hot path) through
the library's async C entry point, input resident in HBM.

Default workload: skewed_1g, n = 2^30 uint32, byte lengths with
P = (.50, .30, .15, .05), values uniform within each length (seeded,
synthetic: the paper's ClueWeb09 posting lists are not available).  Its 2 GiB
stream and 4 GiB output are far larger than L2, so no flush is needed between
steps.

Prints one JSON line (rank 0).  Also reported in the same line:
  roofline      decode kernel's algorithmic bytes / CUDA-event time vs the
                measured HBM copy bandwidth
  e2e           the same metric through svb_decode_host (host buffers, the
                copies in and out inside the timed region)
  cpu_baseline  the oracle (plain scalar C) on a bounded sample, on all host
                cores (a chunked harness) and on one core
  secondary     the delta_64m workload (delta decode and encode) and the
                encoder on skewed_1g, each with its roofline fraction

--impl reference times the oracle on the host cores instead (the paper's
method as a plain scalar program; there is no other implementation to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="skewed_1g")
    ap.add_argument("--n", type=int, default=0, help="decode only the first n integers")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-lists", action="store_true", help="skip the batched-lists workload")
    ap.add_argument("--list-count", type=int, default=100_000)
    return ap.parse_args()


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def code_only(src: str) -> str:
    """C/CUDA source without its comments and with whitespace collapsed, so
    that an edit of comments or layout leaves the hash of the code as it is."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash() -> str:
    """Hash of the code (comments and layout aside) of the sources the decode
    kernels are built from."""
    h = hashlib.sha256()
    for f in ("svb_decode_tiled.cu", "svb_quad.cuh", "svb_device.cuh", "svb_subtile.cuh"):
        src = open(os.path.join(ROOT, "paper_1709_08990_gb300", "csrc", f)).read()
        h.update(code_only(src).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str) -> int | None:
    """DRAM bytes (read + write) per launch of `kernel` on `workload`, from
    the committed ncu summary profiles/traffic.txt, when the summary was taken
    on the current kernel sources (else None).  Line format:
    kernel workload bytes_per_launch source_hash"""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload \
                and f[3] == src:
            return int(f[2])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = open(os.devnull if False else "/tmp/svb_clocks.csv", "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.out:
            self.out.close()

    def summary(self) -> dict:
        try:
            rows = [l.strip().split(", ") for l in open("/tmp/svb_clocks.csv") if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_decode_rate(stream: np.ndarray, n: int, delta: bool, seconds: float):
    """Oracle decode of one sample, repeated for about `seconds`; Gints/s."""
    import oracle
    c = oracle.codec()
    out = np.empty(n, dtype=np.uint32)
    reps, t0 = 0, time.perf_counter()
    while True:
        if delta:
            k = c.lib.svb_ref_delta_decode(stream.ctypes.data, stream.size, n, out.ctypes.data, 0)
        else:
            k = c.lib.svb_ref_decode(stream.ctypes.data, stream.size, n, out.ctypes.data)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    assert k == stream.size
    return reps * n / el / 1e9, reps, el


def oracle_decode_rate_parallel(stream: np.ndarray, n: int, delta: bool, seconds: float,
                                threads: int):
    """The oracle's decoder on `threads` host threads (a chunked harness that
    calls the oracle for every byte count and integer), repeated for about
    `seconds`; Gints/s."""
    import oracle
    par = oracle.parallel()
    out = np.empty(n, dtype=np.uint32)
    reps, t0 = 0, time.perf_counter()
    while True:
        _, k = par.decode(stream, n, delta=delta, threads=threads, out=out)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    assert k == stream.size
    return reps * n / el / 1e9, reps, el


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def reference_arm(args, rank: int):
    """The oracle timed on the host cores, K steps of a bounded sample."""
    if rank != 0:
        return
    from paper_1709_08990_gb300 import workloads as W
    import oracle
    w = W.WORKLOADS[args.workload]
    # About 60 s of oracle work over all K steps (it decodes ~0.1 Gints/s).
    m = 1 << 24
    while m > (1 << 16) and args.steps * m > 6_000_000_000:
        m >>= 1
    x = W.array_values(args.workload, n=m)
    s = oracle.encode(x, delta=w.delta)
    cores = host_cores()
    par = oracle.parallel()
    out = np.empty(m, dtype=np.uint32)

    def fn():
        par.decode(s, m, delta=w.delta, threads=cores, out=out)

    for _ in range(args.warmup):
        fn()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn()
    el = time.perf_counter() - t0
    assert np.array_equal(out, x)
    value = args.steps * m / el / 1e9
    sample = (f"first {m} integers of {args.workload}, decoded {args.steps} times by the "
              f"oracle on {cores} host threads (chunked harness)")
    line = {
        "impl": "reference", "metric": "decode_gints_per_s", "value": value, "unit": "Gints/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "n": m, "delta": w.delta},
        "cpu_baseline": {"value": value, "unit": "Gints/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gints/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate_replicas(total_ms: float, ints_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job timing of N replicas: the longest rank's timed region (each
    rank decodes its own copy of the workload, no data-path collective) and
    the rate of all ranks' integers over it, in Gints/s.  dist is
    torch.distributed with an initialised process group, or None for one
    process."""
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, ints_per_rank * steps * world / (total_ms / 1e3) / 1e9


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    from paper_1709_08990_gb300 import svb
    from paper_1709_08990_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    dev = torch.device("cuda", local)
    w = W.WORKLOADS[args.workload]
    n = args.n if args.n else w.n
    peaks = measured_peaks()

    # ---- inputs: values on the host (seeded), encoded on the device --------
    h_x = torch.empty(n, dtype=torch.int32, pin_memory=True)
    W.array_values(args.workload, n=n, out=h_x.numpy().view(np.uint32))
    d_x = h_x.to(dev, non_blocking=True)
    torch.cuda.synchronize()
    d_stream = svb.encode(d_x, delta=w.delta)
    in_len = d_stream.numel()
    d_out = torch.empty(n, dtype=torch.int32, device=dev)
    ws_bytes = svb.svb_workspace_size(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    svb.svb_workspace_init(ws, ws_bytes, stream)

    def step():
        st = svb.svb_decode_async(d_stream, in_len, n, d_out, 0, int(w.delta), res, ws, ws_bytes,
                                  stream)
        if st != 0:
            raise RuntimeError(f"decode launch failed: {st}")

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    if r[1] != 0 or r[0] != in_len or not torch.equal(d_out, d_x):
        raise RuntimeError("decode result differs from the encoded values")
    del d_x

    # ---- timed region: K decodes, events per launch ---------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    total_ms, value = aggregate_replicas(t_start.elapsed_time(t_end), n, args.steps, dist, dev)
    step_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    alg_bytes = in_len + 4 * n  # control + data read, 4n written

    # Per-kernel times, live: a second pass of the same K steps with the
    # library's CUDA-event bracketing on (each launch timed on its stream).
    svb.svb_profile_begin()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kernels = svb.profile_end()
    top = max(kernels, key=lambda k: kernels[k][1])
    top_ms = kernels[top][1] / kernels[top][0]
    achieved = alg_bytes / (top_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                "kernel": top, "kernel_ms": top_ms, "alg_bytes_per_launch": alg_bytes,
                "alg_bytes_note": "control + data bytes read + 4n bytes written per decode",
                "step_ms": step_ms,
                "step_frac": alg_bytes / (step_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                "traffic": ncu_traffic(top, args.workload)}

    line = {
        "metric": "decode_gints_per_s", "value": value, "unit": "Gints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "delta": w.delta, "stream_bytes": in_len,
                   "bits_per_int": 8.0 * in_len / n, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": roofline,
        "kernels": {k: {"launches": c, "ms_per_launch": t / c} for k, (c, t) in kernels.items()},
        "clocks": clocks.summary(),
        "gpu_launches": args.steps * sum(c for c, _ in kernels.values()) // max(1, args.steps),
    }

    # ---- e2e: through the host-buffer C entry point ----------------------
    if not args.no_e2e:
        h_stream = torch.empty(in_len, dtype=torch.uint8, pin_memory=True)
        h_stream.copy_(d_stream)
        h_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
        d_in2 = torch.empty(in_len, dtype=torch.uint8, device=dev)
        k_e2e = max(3, min(10, args.steps))
        # Untimed warm-up, as for the device-timed steps: at least W calls,
        # then on until two calls in a row agree within 2 % (the first
        # host-buffer calls after the device-timed region can run several
        # times slower), 20 calls at most.
        warm = []
        while len(warm) < 20:
            t0 = time.perf_counter()
            svb.svb_decode_host(h_stream, in_len, n, h_out, 0, int(w.delta), d_in2, d_out)
            warm.append(time.perf_counter() - t0)
            if len(warm) >= max(1, args.warmup) and len(warm) >= 2 and \
                    abs(warm[-1] - warm[-2]) <= 0.02 * min(warm[-1], warm[-2]):
                break
        torch.cuda.synchronize()
        barrier()
        per_step = []
        for _ in range(k_e2e):
            t0 = time.perf_counter()
            svb.svb_decode_host(h_stream, in_len, n, h_out, 0, int(w.delta), d_in2, d_out)
            per_step.append(time.perf_counter() - t0)
        el = sum(per_step)
        barrier()
        ok = torch.equal(h_out, h_x)
        # The host link's floor for this step: the same copy in and copy out,
        # at the same time on two streams, with no decode.
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        t_link = []
        for _ in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            with torch.cuda.stream(s_in):
                d_in2.copy_(h_stream, non_blocking=True)
            with torch.cuda.stream(s_out):
                h_out.copy_(d_out, non_blocking=True)
            torch.cuda.synchronize()
            t_link.append(time.perf_counter() - t1)
        line["e2e"] = {"value": n * k_e2e * world / el / 1e9, "unit": "Gints/s",
                       "h2d_bytes_per_step": in_len, "d2h_bytes_per_step": 4 * n + 16,
                       "steps": k_e2e, "verified": bool(ok), "ms_per_step": el / k_e2e * 1e3,
                       "ms_per_step_min": min(per_step) * 1e3,
                       "ms_per_step_median": float(np.median(per_step)) * 1e3,
                       "ms_each_step": [round(t * 1e3, 3) for t in per_step],
                       "ms_each_warmup_call": [round(t * 1e3, 3) for t in warm],
                       "copies_alone_ms": min(t_link) * 1e3,
                       "note": "copies overlap the decode; copies_alone_ms is the same two "
                               "copies at once with no decode (the host link's floor)"}
        del d_in2, h_out, h_stream

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1) ---------
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        m = 1 << 25
        xs = h_x.numpy().view(np.uint32)[:m]
        s = oracle.encode(xs, delta=w.delta)
        cores = host_cores()
        rate1, reps1, el1 = oracle_decode_rate(s, m, w.delta, args.cpu_seconds / 2)
        rate, reps, el = oracle_decode_rate_parallel(s, m, w.delta, args.cpu_seconds / 2, cores)
        line["cpu_baseline"] = {
            "value": rate, "unit": "Gints/s", "cores": cores, "kind": "oracle",
            "single_core_value": rate1,
            "sample": f"first 2^25 integers of {args.workload}: {reps} decodes on {cores} "
                      f"threads in {el:.1f} s (chunked harness around the oracle), "
                      f"{reps1} on one core in {el1:.1f} s"}

    # ---- secondary workloads --------------------------------------------------
    if not args.no_secondary:
        sec = {}
        svb.svb_set_decode_variant(svb.SVB_DECODE_SINGLE_PASS)
        ms1 = _time(step, 50, stream)
        svb.svb_set_decode_variant(svb.SVB_DECODE_AUTO)
        ok1 = torch.equal(d_out[:1 << 20], h_x[:1 << 20].to(dev))
        sec["decode_single_pass_" + args.workload] = {
            "gints_per_s": n / ms1 / 1e6, "ms": ms1, "frac": alg_bytes / (ms1 / 1e3) / 1e9 /
            peaks["hbm_gbs"], "verified_prefix": bool(ok1)}
        if not w.delta:   # the chunked single pass decodes plain streams
            d_out.zero_()
            svb.svb_set_decode_variant(svb.SVB_DECODE_CHUNKED)
            ms5 = _time(step, 50, stream)
            svb.svb_set_decode_variant(svb.SVB_DECODE_AUTO)
            ok5 = torch.equal(d_out[:n], h_x.to(dev))
            sec["decode_chunked_" + args.workload] = {
                "gints_per_s": n / ms5 / 1e6, "ms": ms5,
                "frac": alg_bytes / (ms5 / 1e3) / 1e9 / peaks["hbm_gbs"], "verified": bool(ok5)}
        del d_out, d_stream
        torch.cuda.empty_cache()
        sec["encode_" + args.workload] = time_encode(svb, W, args.workload, dev, peaks, h_x)
        del h_x
        sec["delta_64m"] = time_codec(svb, W, "delta_64m", dev, peaks)
        sec["uniform_1m"] = time_codec(svb, W, "uniform_1m", dev, peaks)
        sec["seek_select_256"] = time_queries(svb, dev)
        sec["append"] = time_append(svb, W, dev)
        if not args.no_lists:
            torch.cuda.empty_cache()
            sec["lists_100k"] = time_lists(svb, W, dev, peaks, args.list_count)
            sec["lists_1000_unscaled"] = time_long_lists(svb, W, dev, peaks)
        line["secondary"] = sec

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _time(fn, steps, stream):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def time_encode(svb, W, name, dev, peaks, h_x):
    import torch
    n = h_x.numel()
    d_x = h_x.to(dev)
    d_s = torch.empty(svb.svb_max_compressed_size(n), dtype=torch.uint8, device=dev)
    ws_bytes = svb.svb_workspace_size(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    svb.svb_workspace_init(ws, ws_bytes, stream)
    delta = W.WORKLOADS[name].delta
    ms = _time(lambda: svb.svb_encode_async(d_x, n, d_s, 0, int(delta), res, ws, ws_bytes, stream),
               50, stream)
    size = int(res[0].item())
    alg = 4 * n + size
    out = {"gints_per_s": n / ms / 1e6, "ms": ms, "frac": alg / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
           "alg_bytes": alg}
    del d_s, ws
    torch.cuda.empty_cache()
    out["size_report"] = time_size_report(svb, d_x, delta, peaks)
    # The paper's reference line: copying the uncompressed integers (memcpy).
    d_y = torch.empty_like(d_x)
    ms_c = _time(lambda: d_y.copy_(d_x), 20, stream)
    out["memcpy_4n"] = {"gints_per_s": n / ms_c / 1e6, "ms": ms_c,
                        "gb_per_s": 8 * n / (ms_c / 1e3) / 1e9}
    del d_x, d_y
    torch.cuda.empty_cache()
    return out


def time_size_report(svb, d_x, delta, peaks):
    """Stream VByte and VByte sizes (Sec. 5, Fig. 5b) of the resident values,
    and the size kernel's own read bandwidth (4n bytes per call)."""
    import torch
    n = d_x.numel()
    s_svb, s_vb = svb.size_report(d_x, delta=delta)
    d = torch.zeros(2, dtype=torch.int64, device=d_x.device)
    stream = torch.cuda.current_stream()
    ms = _time(lambda: svb.svb_size_report_async(d_x, n, 0, int(delta), d, stream), 50, stream)
    return {"svb_bits_per_int": 8.0 * s_svb / n, "vbyte_bits_per_int": 8.0 * s_vb / n,
            "extra_bits_per_int": 8.0 * (s_svb - s_vb) / n, "ms": ms,
            "frac": 4 * n / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}


def time_codec(svb, W, name, dev, peaks):
    import torch
    w = W.WORKLOADS[name]
    x = W.array_values(name)
    d_x = torch.from_numpy(x.view(np.int32)).to(dev)
    n = x.size
    d_s = torch.empty(svb.svb_max_compressed_size(n), dtype=torch.uint8, device=dev)
    d_o = torch.empty(n, dtype=torch.int32, device=dev)
    ws_bytes = svb.svb_workspace_size(n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    svb.svb_workspace_init(ws, ws_bytes, stream)
    steps = 200 if n > (1 << 22) else 2000
    ms_e = _time(lambda: svb.svb_encode_async(d_x, n, d_s, 0, int(w.delta), res, ws, ws_bytes, stream),
                 steps, stream)
    size = int(res[0].item())
    ms_d = _time(lambda: svb.svb_decode_async(d_s, size, n, d_o, 0, int(w.delta), res, ws, ws_bytes,
                                              stream), steps, stream)
    ok = torch.equal(d_o, d_x)
    alg = 4 * n + size
    hb = peaks["hbm_gbs"]
    extra = {}
    if w.delta:
        # The three-launch form (offsets pass, sums pass over staged tiles,
        # decode) beside the default one-pass offsets and carries.
        svb.svb_set_decode_variant(svb.SVB_DECODE_SUMS_PASS)
        ms_3 = _time(lambda: svb.svb_decode_async(d_s, size, n, d_o, 0, 1, res, ws, ws_bytes,
                                                  stream), steps, stream)
        svb.svb_set_decode_variant(svb.SVB_DECODE_AUTO)
        ok = ok and torch.equal(d_o, d_x)
        extra["decode_sums_pass"] = {"gints_per_s": n / ms_3 / 1e6, "us": ms_3 * 1e3,
                                     "frac": alg / (ms_3 / 1e3) / 1e9 / hb}
    s_svb, s_vb = svb.size_report(d_x, delta=w.delta)
    return {**extra, "n": n, "delta": w.delta, "stream_bytes": size, "verified": bool(ok),
            "bits_per_int": {"svb": 8.0 * s_svb / n, "vbyte": 8.0 * s_vb / n,
                             "extra": 8.0 * (s_svb - s_vb) / n},
            "decode": {"gints_per_s": n / ms_d / 1e6, "us": ms_d * 1e3,
                       "frac": alg / (ms_d / 1e3) / 1e9 / hb},
            "encode": {"gints_per_s": n / ms_e / 1e6, "us": ms_e * 1e3,
                       "frac": alg / (ms_e / 1e3) / 1e9 / hb}}


def time_queries(svb, dev, num_lists: int = 1 << 20, nq: int = 1 << 22):
    """Seek and select (Sec. 5, Fig. 6) in the paper's setting: lists of 256
    integers whose deltas are uniform in [0, 2^b), prefix-summed and
    differentially coded; queries pick a list uniformly, seek targets are
    uniform in [0, the list's last integer], select indexes uniform in
    [0, 256).  One launch answers all queries; reported as queries/s."""
    import torch
    from paper_1709_08990_gb300.batch import ListPool
    out = {"lists": num_lists, "list_len": 256, "queries": nq}
    for bits in (8, 24):
        rng = np.random.default_rng(600 + bits)
        d = rng.integers(0, 1 << bits, (num_lists, 256), dtype=np.uint64)
        vals = (np.cumsum(d, axis=1) & 0xFFFFFFFF).astype(np.uint32)
        lengths = np.full(num_lists, 256, dtype=np.uint32)
        pool = ListPool(lengths, vals.reshape(-1), delta=True, device=dev)
        res = {"pool_bytes": pool.pool_bytes}
        d_tab = torch.from_numpy(pool.dec_table.view(np.uint8).copy()).to(dev)
        for op in (svb.SVB_SEEK, svb.SVB_SELECT):
            q = np.zeros(nq, dtype=svb.query_dtype())
            q["list"] = rng.integers(0, num_lists, nq)
            q["op"] = op
            if op == svb.SVB_SEEK:
                last = vals[q["list"], -1].astype(np.uint64)
                q["arg"] = (rng.random(nq) * (last + 1)).astype(np.uint64)
            else:
                q["arg"] = rng.integers(0, 256, nq)
            d_q = torch.from_numpy(q.view(np.uint8).copy()).to(dev)
            d_a = torch.zeros(nq * svb.answer_dtype().itemsize, dtype=torch.uint8, device=dev)
            stream = torch.cuda.current_stream()
            ms = _time(lambda: svb.svb_query_batch(d_tab, num_lists, pool.pool, 1, d_q, nq, d_a,
                                                   stream), 20, stream)
            a = d_a.cpu().numpy().view(svb.answer_dtype())
            # spot-check against the decoded lists
            k = rng.integers(0, nq, 256)
            ok = bool(np.all(a["status"][k] == 0))
            for i in k:
                li, arg = int(q["list"][i]), int(q["arg"][i])
                row = vals[li]
                if op == svb.SVB_SEEK:
                    j = int(np.searchsorted(row, arg, side="left"))
                    ok &= int(a["index"][i]) == j and (j == 256 or int(a["value"][i]) == int(row[j]))
                else:
                    ok &= int(a["value"][i]) == int(row[arg])
            res["seek" if op == svb.SVB_SEEK else "select"] = {
                "mqueries_per_s": nq / ms / 1e3, "ms": ms, "verified_sample": bool(ok)}
        out[f"b{bits}"] = res
        del pool, d_tab
        torch.cuda.empty_cache()
    return out


def time_append(svb, W, dev, n0: int = 1 << 26, k: int = 1 << 20):
    """Appending k integers to an n0-integer compressed array (Sec. 4's
    closing remark) against encoding all n0 + k from scratch; skewed values."""
    import torch
    x = W.array_values("skewed_1g", n=n0 + k)
    d_x = torch.from_numpy(x.view(np.int32)).to(dev)
    s = svb.encode(d_x[:n0])
    nc = (n0 + 3) // 4
    ctrl_cap, data_cap = (n0 + k + 3) // 4 + 8, s.numel() - nc + 4 * k + 64
    d_ctrl = torch.zeros(ctrl_cap, dtype=torch.uint8, device=dev)
    d_data = torch.zeros(data_cap, dtype=torch.uint8, device=dev)
    d_ctrl0 = s[:nc].clone()
    d_data0 = s[nc:].clone()
    data_len0 = s.numel() - nc
    d_new = d_x[n0:]
    reps = 20
    torch.cuda.synchronize()
    t = 0.0
    for i in range(reps + 3):
        d_ctrl[:nc].copy_(d_ctrl0)          # restore the n0-integer array (untimed)
        d_data[:data_len0].copy_(d_data0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dl = svb.svb_append(d_ctrl, ctrl_cap, d_data, data_cap, data_len0, n0, d_new, k, 0, 0)
        el = time.perf_counter() - t0
        if i >= 3:
            t += el
    ms = t / reps * 1e3
    whole = svb.encode(d_x)
    ok = bool(torch.equal(d_ctrl[:(n0 + k + 3) // 4], whole[:(n0 + k + 3) // 4])) and \
        bool(torch.equal(d_data[:dl], whole[(n0 + k + 3) // 4:]))
    ws = torch.empty(svb.svb_workspace_size(n0 + k), dtype=torch.uint8, device=dev)
    res = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    svb.svb_workspace_init(ws, ws.numel(), stream)
    out = torch.empty(svb.svb_max_compressed_size(n0 + k), dtype=torch.uint8, device=dev)
    ms_enc = _time(lambda: svb.svb_encode_async(d_x, n0 + k, out, 0, 0, res, ws, ws.numel(),
                                                stream), 10, stream)
    return {"n0": n0, "k": k, "append_ms": ms, "append_gints_per_s": k / ms / 1e6,
            "reencode_all_ms": ms_enc, "verified": ok,
            "note": "append timed on the host around the synchronous call"}


def time_serve(pool, W, seconds: float = 1.0, peak_requests: int = 400_000,
               level_cap: int = 200_000):
    """Serving loop over the pool: peak throughput with peak_requests queued
    at once (tens of batches), then Poisson arrivals offering 10%..90% of that
    peak in integers per second: each level's requests are drawn first and
    their arrival rate set from their own mean size, for about `seconds` or
    level_cap requests, whichever is fewer (the fresh lists of a level's
    encode requests live in host memory)."""
    from paper_1709_08990_gb300.serve import Server, summarize
    srv = Server(pool, budget=16 << 30)
    warm = W.serve_requests(pool.lengths, 20_000, None, seed=105)
    srv.run(warm)
    req = W.serve_requests(pool.lengths, peak_requests, None, seed=5)
    peak = summarize(req, srv.run(req))
    del req
    peak_ints = peak["gints_per_s"] * 1e9
    mean_n = peak["ints"] / peak["requests"]
    levels = []
    for i, f in enumerate([0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9]):
        count = min(level_cap, max(2000, int(seconds * f * peak_ints / mean_n)))
        r = W.serve_requests(pool.lengths, count, 1.0, seed=5 + 1000 * (i + 1))
        rate = f * peak_ints / float(r.n.mean())    # requests/s offering f x peak ints/s
        r.arrival = r.arrival / rate
        s = summarize(r, srv.run(r))
        s["load"] = f
        s["offered_gints_per_s"] = rate * float(r.n.mean()) / 1e9
        s["offered_frac_of_peak"] = s["offered_gints_per_s"] * 1e9 / peak_ints
        s["achieved_frac_of_offered"] = s["gints_per_s"] / s["offered_gints_per_s"]
        s["window_s"] = float(r.arrival[-1])
        levels.append(s)
    return {"budget_bytes": 16 << 30, "slots": len(srv.slots), "max_batch": srv.max_batch,
            "mean_request_ints": mean_n, "peak": peak, "levels": levels}


serve_levels = True


def time_lists(svb, W, dev, peaks, count: int):
    """Batched delta decode/encode of the lists_100k workload (one persistent
    launch, replayed from a CUDA graph) against one call per list: from a
    Python loop, from the library's host loop, and that loop replayed from a
    CUDA graph."""
    import torch
    from paper_1709_08990_gb300 import autotune
    from paper_1709_08990_gb300.batch import ListPool
    L = W.lists_lengths(count, cap=(1 << 30) * count // 100_000)
    h_vals = torch.empty(int(L.sum()), dtype=torch.int32, pin_memory=True)
    W.posting_lists(W.WORKLOADS["lists_100k"].seed, L, out=h_vals.numpy().view(np.uint32))
    d_vals = h_vals.to(dev)
    pool = ListPool(L, d_vals, delta=True, device=dev)
    total = pool.total
    d_out = torch.empty(total, dtype=torch.int32, device=dev)
    d_enc = torch.empty_like(pool.pool)
    tuned = autotune.tune_batch(pool, f"lists_{count}", d_out, enc_out=d_enc)
    stream = torch.cuda.current_stream()
    g = pool.graph(lambda: pool.decode(d_out))
    ms_graph = _time(lambda: g.replay(), 20, stream)
    ms_batch = _time(lambda: pool.decode(d_out), 20, stream)
    r = pool.result()
    ok = bool(r[1] == 0 and torch.equal(d_out, d_vals))
    # One launch per list, every list once.
    d_out2 = torch.zeros_like(d_out)
    ws = pool.decode_per_list(d_out2, lists=range(min(64, pool.k)))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pool.decode_per_list(d_out2, ws=ws)
    b.record(stream)
    torch.cuda.synchronize()
    ms_per_list = a.elapsed_time(b)
    ok_per_list = bool(torch.equal(d_out2, d_vals))
    # Encode: batched vs per list.
    d_enc = torch.empty(pool.pool_bytes, dtype=torch.uint8, device=dev)
    ms_benc = _time(lambda: pool.encode(d_enc), 10, stream)
    ok_enc = bool(torch.equal(d_enc, pool.pool))
    a.record(stream)
    pool.encode_per_list(d_enc, ws=ws)
    b.record(stream)
    torch.cuda.synchronize()
    ms_enc_per_list = a.elapsed_time(b)
    # One call per list issued by the library's own host loop (no interpreter
    # between launches), eager and captured once into a CUDA graph.
    ews = pool.each_workspace()
    d_res = torch.zeros(2 * pool.k, dtype=torch.int64, device=dev)
    d_out3 = torch.zeros_like(d_out)
    pool.decode_each(d_out3, ews, d_res)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.record(stream)
    pool.decode_each(d_out3, ews, d_res)
    b.record(stream)
    host_ms_each = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()
    ms_each = a.elapsed_time(b)
    ok_each = bool(torch.equal(d_out3, d_vals)) and int(d_res.view(-1, 2)[:, 1].max()) == 0
    a.record(stream)
    pool.encode_each(d_enc, ews, d_res)
    b.record(stream)
    torch.cuda.synchronize()
    ms_enc_each = a.elapsed_time(b)
    ok_enc_each = bool(torch.equal(d_enc, pool.pool))
    each_graph = {}
    try:
        gd = pool.graph(lambda: pool.decode_each(d_out3, ews, d_res))
        ms_each_graph = _time(lambda: gd.replay(), 3, stream)
        ok_g = bool(torch.equal(d_out3, d_vals))
        del gd
        ge = pool.graph(lambda: pool.encode_each(d_enc, ews, d_res))
        ms_enc_each_graph = _time(lambda: ge.replay(), 3, stream)
        ok_ge = bool(torch.equal(d_enc, pool.pool))
        del ge
        each_graph = {
            "decode_per_list_graph": {"gints_per_s": total / ms_each_graph / 1e6,
                                      "ms": ms_each_graph, "verified": ok_g},
            "decode_speedup_vs_per_list_graph": ms_each_graph / ms_graph,
            "encode_per_list_graph": {"gints_per_s": total / ms_enc_each_graph / 1e6,
                                      "ms": ms_enc_each_graph, "verified": ok_ge},
            "encode_speedup_vs_per_list_graph": ms_enc_each_graph / ms_benc}
    except RuntimeError as e:  # capture of ~2 launches per list may not fit
        each_graph = {"per_list_graph_error": str(e)[:200]}
    del ews, d_res, d_out3
    alg = pool.pool_bytes + 4 * total
    hb = peaks["hbm_gbs"]
    serve = time_serve(pool, W) if serve_levels else None
    out = {"lists": pool.k, "ints": total, "stream_bytes": pool.pool_bytes,
           "min_len": int(L.min()), "max_len": int(L.max()),
           "not_multiple_of_4": int((L % 4 != 0).sum()), "verified": ok and ok_per_list and ok_enc,
           "tuned": {"threshold": tuned["threshold"], "grid": tuned["grid"],
                     "segment_tiles": tuned.get("segment_tiles"),
                     "stages": tuned.get("stages"), "tile_ints": tuned.get("tile_ints"),
                     "encode_threshold": tuned.get("encode_threshold"),
                     "encode_stages": tuned.get("encode_stages"), "cached": tuned["cached"]},
           "decode_batched_graph": {"gints_per_s": total / ms_graph / 1e6, "ms": ms_graph,
                                    "frac": alg / (ms_graph / 1e3) / 1e9 / hb},
           "decode_batched_launch": {"gints_per_s": total / ms_batch / 1e6, "ms": ms_batch},
           "decode_per_list": {"gints_per_s": total / ms_per_list / 1e6, "ms": ms_per_list},
           "decode_speedup_vs_per_list": ms_per_list / ms_graph,
           "decode_per_list_c_loop": {"gints_per_s": total / ms_each / 1e6, "ms": ms_each,
                                      "host_issue_ms": host_ms_each, "verified": ok_each},
           "decode_speedup_vs_per_list_c_loop": ms_each / ms_graph,
           "encode_per_list_c_loop": {"gints_per_s": total / ms_enc_each / 1e6,
                                      "ms": ms_enc_each, "verified": ok_enc_each},
           "encode_speedup_vs_per_list_c_loop": ms_enc_each / ms_benc,
           **each_graph,
           "encode_batched": {"gints_per_s": total / ms_benc / 1e6, "ms": ms_benc,
                              "frac": alg / (ms_benc / 1e3) / 1e9 / hb},
           "encode_per_list": {"gints_per_s": total / ms_enc_per_list / 1e6,
                               "ms": ms_enc_per_list},
           "encode_speedup_vs_per_list": ms_enc_per_list / ms_benc,
           "serve": serve}
    del pool, d_out, d_out2, d_enc, d_vals
    torch.cuda.empty_cache()
    return out


def time_long_lists(svb, W, dev, peaks, count: int = 1000):
    """The list workload's lengths unscaled (log-uniform up to 4,194,304
    integers): one batched decode with long lists cut into units decoded by
    several CTAs, against the same batch with every big list decoded whole."""
    import torch
    from paper_1709_08990_gb300.batch import ListPool
    L = W.lists_lengths(count, cap=1 << 40)
    h = np.empty(int(L.sum()), dtype=np.uint32)
    W.posting_lists(W.WORKLOADS["lists_100k"].seed, L, out=h)
    d_vals = torch.from_numpy(h.view(np.int32)).to(dev)
    del h
    pool = ListPool(L, d_vals, delta=True, device=dev)
    total = pool.total
    d_out = torch.empty(total, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"lists": pool.k, "ints": total, "max_len": int(L.max()),
           "stream_bytes": pool.pool_bytes}
    alg = pool.pool_bytes + 4 * total
    for name, seg in (("split", None), ("whole", 0)):
        pool.replan(pool.threshold, 0, seg)
        d_out.zero_()
        g = pool.graph(lambda: pool.decode(d_out))
        ms = _time(lambda: g.replay(), 20, stream)
        ok = bool(pool.result()[1] == 0 and torch.equal(d_out, d_vals))
        out[name] = {"gints_per_s": total / ms / 1e6, "ms": ms, "verified": ok,
                     "frac": alg / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
        del g
    out["speedup_split_vs_whole"] = out["whole"]["ms"] / out["split"]["ms"]
    del pool, d_out, d_vals
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
