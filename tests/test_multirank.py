"""The N > 1 host logic of bench.py (replicas: no collective on the data path)
on two gloo ranks on the CPU: the step time is the slowest rank's, and the job
value counts every replica's bytes over it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank_ms(torch, dist, [10.0, 12.5][rank], device="cpu")
        dist.barrier()
        out[rank] = ms
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 12.5
    # 2 replicas x 1 GB each in 12.5 ms
    assert bench.replica_value(world, 1e9, out[0]) == pytest.approx(160.0)


def test_single_process_keeps_its_own_time():
    assert bench.slowest_rank_ms(torch, None, 7.0) == 7.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the oracle arm is timed by rank 0; other ranks return at once."""
    monkeypatch.setenv("RANK", "1")
    args = bench.parse_args_for_test(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) is None


def test_all_core_oracle_baseline_runs_spawned_replicas():
    """The all-core CPU baseline: single-threaded oracle processes from a spawn
    pool, timed from their common start."""
    r = bench.cpu_baseline_all_cores(4, 1, steps=1, max_procs=2)
    assert r["cores"] <= 2 and r["value"] > 0 and r["seconds"] > 0
