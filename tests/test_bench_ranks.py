"""Multi-rank host logic of bench.py on the CPU: two gloo ranks, as torchrun
launches them (one process per GPU). The path shards into replicas, each rank
with its own seeded instance and no exchange; the line reports the slowest rank's
time and the units of all ranks over it."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = [0.20, 0.35][rank]  # per-step time of this rank
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    e2e = bench.max_over_ranks([1.5, 1.25][rank], dist, device="cpu")
    q.put((rank, slowest, e2e, bench.aggregate_rate(world, 1000, slowest),
           bench.replica_seed(2, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, e2e, rate, seed in out:
        assert slowest == pytest.approx(0.35)
        assert e2e == pytest.approx(1.5)
        assert rate == pytest.approx(2 * 1000 / 0.35e-3)
    assert out[0][4] != out[1][4]  # independent replicas


def test_single_process_needs_no_collective():
    import bench

    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.aggregate_rate(1, 1000, 0.5) == pytest.approx(2e6)
