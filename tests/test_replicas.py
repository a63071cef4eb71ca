"""The multi-replica path of bench.py on CPU: two gloo ranks each time their
own copy of the workload; the job's time is the longest rank's and its rate
counts every rank's integers.  Runs without a GPU (world size 2, 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r's timed region took 10 (r + 1) ms for 1000 integers x 5 steps
        total_ms, value = bench.aggregate_replicas(10.0 * (rank + 1), 1000, 5, dist, "cpu")
        out[rank] = (total_ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_longest_time_and_count_all_integers():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    want_ms = 20.0
    want_value = 1000 * 5 * world / (want_ms / 1e3) / 1e9
    for r in range(world):
        total_ms, value = res[r]
        assert total_ms == pytest.approx(want_ms)
        assert value == pytest.approx(want_value)


def test_one_process_needs_no_process_group():
    total_ms, value = bench.aggregate_replicas(4.0, 1 << 20, 10)
    assert total_ms == 4.0
    assert value == pytest.approx((1 << 20) * 10 / 4e-3 / 1e9)
