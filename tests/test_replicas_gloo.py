"""Multi-GPU runs of this solver are independent replicas (one solve per rank, no data-path
collective).  The only cross-rank step is the benchmark's aggregation: the slowest rank's
time and the sum of all ranks' work.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, flops = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 1e12 * (rank + 1))
        out[rank] = (ms, flops)
    finally:
        tdist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
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
            assert out[r] == pytest.approx((150.0, 3e12))


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_over_ranks(12.5, 7.0) == (12.5, 7.0)
