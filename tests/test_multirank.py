"""Host logic of the multi-GPU benchmark on CPU: two gloo ranks.

Slices are independent problems, so ranks share no data: the cross-rank steps
are the max over ranks of the timed region, from which the whole-job
throughput (all ranks' slice-iterations over the slowest rank's time) follows,
and the host gather of the per-slice results on rank 0 after the batched
workload was partitioned over the ranks (balanced by pixels x iterations).
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


def test_partition_is_balanced_and_covers_every_slice_once():
    import bench
    import numpy as np
    rng = np.random.default_rng(0)
    # the mixed workload's costs (pixels x iterations) and random ones
    mixed = [128 * 128 * 30] * 32 + [256 * 256 * 30] * 32 + [384 * 320 * 30] * 32
    for costs in (mixed, [320 * 320 * 20] * 256, list(rng.integers(1, 1000, 77))):
        for world in (1, 2, 3, 8):
            parts = bench.partition_slices(costs, world)
            flat = sorted(i for q in parts for i in q)
            assert flat == list(range(len(costs)))
            loads = [sum(costs[i] for i in q) for q in parts]
            assert max(loads) - min(loads) <= max(costs)
    assert bench.partition_slices([5] * 256, 8) == [list(range(r, 256, 8)) for r in range(8)]


def _gather_worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    costs = [128 * 128] * 5 + [384 * 320] * 4
    parts = bench.partition_slices(costs, world)
    local = {i: ("slice", i, rank) for i in parts[rank]}
    res = bench.gather_by_slice(parts, world, rank, local, len(costs))
    if rank == 0:
        out["res"] = res
        out["parts"] = parts
    else:
        out[f"none{rank}"] = res is None
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_returns_every_slice_in_order():
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res, parts = out["res"], out["parts"]
    assert [r[1] for r in res] == list(range(9))
    for i, r in enumerate(res):
        assert r[2] == (0 if i in parts[0] else 1)
    assert all(len(q) > 0 for q in parts)
    assert out["none1"] is True
