"""The multi-process side of bench.py, on the CPU with the gloo backend (two ranks): each
replica's times are reduced to their maximum over the ranks, and the job's rate counts
every replica's cells against the slowest replica's time.  (The method has no exchange
between ranks: under torchrun every rank runs an independent replica of the workload.)"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench._dist() == (ws, rank)
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank], "cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == [11.0, 5.0] and res[1] == [11.0, 5.0]


def test_job_rate_counts_all_replicas():
    import bench
    assert bench.job_rate(1, 1000, 10, 2.0) == pytest.approx(5000.0)
    assert bench.job_rate(4, 1000, 10, 2.0) == pytest.approx(20000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the oracle on the host) is rank 0's alone; the
    other ranks return at once without work."""
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=3)) is None
