"""The multi-GPU path of bench.py is replicas only (one lattice per rank, no data-path collective):
the timed region is the maximum over ranks and the whole-job time per solve counts every rank's
solves.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        local = 10.0 + 5.0 * rank  # rank 1 is the slow one
        out[rank] = bench.replica_aggregate(local, 5, world, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_solves():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            total, per_replica, whole_job = out[r]
            assert total == 15.0 and per_replica == 3.0 and whole_job == 1.5


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.replica_aggregate(12.0, 4, 1, None, "cpu") == (12.0, 3.0, 3.0)
