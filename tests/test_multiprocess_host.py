"""The N > 1 path of bench.py on CPU: replicas only, so the only cross-rank step
is the max of the timed region (the job lasts as long as its slowest rank) and the
whole-job throughput counts every rank's replica.  Two gloo ranks, spawned."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [12.5, 20.0][rank]                 # rank 1 is the slow one
        t = bench.max_over_ranks(local, dist, device="cpu")
        out[rank] = (t, bench.job_mlups(1000, 10, world, t * 1e-3))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_both_replicas():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        got = dict(out)
    assert got[0] == got[1]                        # every rank sees the same job time
    t, mlups = got[0]
    assert t == 20.0
    assert mlups == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_mlups(100, 5, 1, 0.5) == pytest.approx(100 * 5 / 0.5 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        steps, warmup, cpu_seconds = 1, 1, 0.1
    bench.run_reference(A(), rank=1, world=2)     # other ranks exit without work or output
    assert capsys.readouterr().out == ""
