"""Multi-GPU runs are independent replicas (one problem per rank, no
data-path collective): the benchmark's whole-job figure is the updates of all
ranks over the slowest rank's time.  Checked here with two gloo ranks on the
CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 150.0][rank]
    updates = [1_000_000, 3_000_000][rank]
    out[rank] = bench.reduce_over_ranks(ms, updates, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            t, u = out[r]
            assert t == 150.0 and u == 4_000_000.0
    # one rank: figures unchanged
    import bench
    assert bench.reduce_over_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)
