"""Host logic of bench.py's multi-GPU form, run as two gloo ranks on the CPU.

The method is run as independent replicas (one lattice per GPU, no data
exchange between them): the whole job's time is the slowest rank's, and its
throughput counts the lattice updates of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup(None)
        assert (w, r, local) == (world, rank, rank)
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slower replica
        worst = bench.max_over_ranks(ms, w, device="cpu")
        out[rank] = (worst, bench.job_rate(1000, w, worst / 1e3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_and_the_whole_job():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    worst, rate = res[0]
    assert worst == 15.0
    assert rate == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
