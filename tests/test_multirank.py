"""Host logic of the multi-GPU benchmark on CPU: two gloo ranks.

Slices are independent problems, so ranks share no data: the only cross-rank
step is the max over ranks of the timed region, from which the whole-job
throughput (all ranks' slice-iterations over the slowest rank's time) follows.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local = [12.5, 20.0][rank]
    m = bench.slowest_rank_ms(local, world)
    v = bench.job_throughput(world, steps=4, iters_per_step=30, slices_per_rank=1, max_ms=m)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        m, v = out[r]
        assert m == 20.0                           # the slowest rank sets the clock
        assert abs(v - 2 * 4 * 30 / 0.020) < 1e-6  # every rank's work over that time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(7.0, 1) == 7.0
    assert bench.job_throughput(1, 10, 30, 1, 1000.0) == 300.0
