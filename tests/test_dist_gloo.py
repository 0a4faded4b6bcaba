"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
step's FP64 MC sums are all-reduced once and added to the running total (the
estimator's only exchange; samples are sharded with no data-path collective),
and the reported time is the slowest rank's."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    acc = torch.zeros(8, dtype=torch.float64)
    step = torch.zeros(8, dtype=torch.float64)
    for k in range(3):                       # three steps of per-rank sums
        step.copy_(torch.arange(8, dtype=torch.float64) * (rank + 1) + k)
        bench.merge_step_sums(dist, step, acc)
    t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, torch.device("cpu"))
    out[rank] = acc.tolist() + [t]
    dist.destroy_process_group()


def test_step_sums_and_max_time_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    expect = [sum(i * (r + 1) + k for r in range(world) for k in range(3)) for i in range(8)]
    for r in range(world):
        assert out[r][:8] == pytest.approx(expect, rel=0, abs=0)
        assert out[r][8] == 15.0


def test_single_process_path_needs_no_group():
    import bench
    acc = torch.zeros(8, dtype=torch.float64)
    bench.merge_step_sums(None, torch.ones(8, dtype=torch.float64), acc)
    bench.merge_step_sums(None, torch.ones(8, dtype=torch.float64), acc)
    assert acc.tolist() == [2.0] * 8
    assert bench.max_over_ranks(None, 3.5, torch.device("cpu")) == 3.5
