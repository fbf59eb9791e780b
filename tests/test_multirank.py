"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) take different timesteps of the same scene,
the timing reduction returns the slowest rank's time on every rank, and the
whole-job rate counts the units of all ranks over that time. No GPU."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        scene = type("S", (), {"n_steps": 300})()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, w, "cpu")
        rate = bench.job_throughput(7 * 20, w, slowest)
        dist.barrier()
        out[rank] = (r, w, local, bench.step_index(scene, r), slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_distinct_timesteps_and_the_slowest_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    steps = {res[r][3] for r in res}
    assert len(steps) == 2                      # one timestep per rank
    for r in res:
        rank, w, local, step, slowest, rate = res[r]
        assert (rank, w, local) == (r, 2, r)
        assert slowest == 15.0                  # max over ranks on every rank
        assert rate == pytest.approx(2 * 7 * 20 / 0.015)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(140, 1, 20.0) == pytest.approx(7000.0)
