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


def test_committed_ncu_records_match_the_kernel_sources():
    # bench.py takes roofline.traffic and roofline_df.traffic (DRAM bytes per launch) from the committed
    # ncu records only while the hashed kernel sources are the ones captured; a source change without a
    # new capture would silently turn those figures into null.  Recapture the record (the command is in
    # the Markdown summary beside it) whenever this fails.
    import bench

    import numpy as np

    vh = int(np.prod(bench.DIMS)) // 2
    fp32 = bench.profiled_traffic("32c8")
    df = bench.profiled_traffic("32c8", record="df_dslash_32c8.json", files=("df64.cu", "common.cuh"))
    # DRAM bytes of one cold launch within 10 % of the algorithmic bytes (no re-reads)
    assert fp32 is not None and abs(fp32 / (bench.DSLASH_BYTES_PER_SITE["fp32"] * vh) - 1) < 0.1
    assert df is not None and abs(df / (bench.DF_BYTES_PER_SITE * vh) - 1) < 0.1
