"""The benchmark's multi-process path on CPU (gloo, world size 2): every rank
solves its own replica (weak scaling, no collective on the data path); the job
time is the maximum over ranks and the job rate counts every rank's units."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1307_3424_gb300 import synth


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_env()
        # each rank times its own replica; rank 1 is the slow one here
        t = [100.0 + 50.0 * r, 120.0 + 10.0 * r]
        t_job = bench.reduce_times_max(t, w)
        # replicas: seed = rank gives each rank its own problem
        prob = synth.make_problem(synth.SMALL, seed=r, M=64)
        out[r] = (w, r, loc, t_job, bench.job_rate(10.5 * 5, w, t_job[0]), float(prob.uvw[0, 0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_count_every_replica():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(worker, args=(ws, free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        w, rank, loc, t_job, rate, u0 = res[r]
        assert (w, rank, loc) == (2, r, r)
        assert t_job == [150.0, 130.0]                  # max over ranks, per timed region
        assert rate == pytest.approx(10.5 * 5 * 2 / 0.150)
    assert res[0][5] != res[1][5]                       # different replicas


def test_single_process_is_a_no_op():
    assert bench.reduce_times_max([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.job_rate(21.0, 1, 1000.0) == pytest.approx(21.0)
