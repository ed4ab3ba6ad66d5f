"""The transport of a domain decomposition across processes (paper_1101_0423_gb300.dist),
checked with gloo ranks on CPU: every face reaches the neighbour on its side as the message
that neighbour expects (its face towards the sender), through the ctypes callbacks the
library calls; and the sums are the same on every rank."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _face(rank, k, n):
    """A face's bytes, telling its sender and index."""
    return (np.arange(n, dtype=np.int64) * 7 + 1000 * rank + k).astype(np.uint8)


def _rank(rank, world, port, grid, out):
    import torch.distributed as tdist

    from paper_1101_0423_gb300 import dist as pdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        coord = pdist.grid_coord(rank, grid)
        assert pdist.grid_rank(coord, grid) == rank
        tc = pdist.TorchPartComm(grid, coord)
        # faces of the cut directions only, sizes differing per direction (as fsz[mu] do)
        nbytes = [(48 * (1 + (k >> 1))) if grid[k >> 1] > 1 else 0 for k in range(8)]
        send = [_face(rank, k, n) if n else None for k, n in enumerate(nbytes)]
        recv = [np.zeros(n, np.uint8) if n else None for n in nbytes]
        # through the C-callable function pointers, as the library calls them
        SP = ctypes.c_void_p * 8
        sp = SP(*[s.ctypes.data if s is not None else None for s in send])
        rp = SP(*[r.ctypes.data if r is not None else None for r in recv])
        nb = (ctypes.c_size_t * 8)(*nbytes)
        rc = tc.comm.exchange(None, sp, rp, nb)
        ok_faces = rc == 0
        for k in range(8):
            if nbytes[k]:
                peer = tc.neighbour(k >> 1, k & 1)
                ok_faces = ok_faces and np.array_equal(recv[k], _face(peer, k ^ 1, nbytes[k]))
        v = np.array([1.5 * (rank + 1), -2.0 ** -30 * rank], dtype=np.float64)
        rc2 = tc.comm.allreduce(None, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2)
        out[rank] = (ok_faces, rc2, v.tolist())
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("grid", [(2, 1, 1, 1), (1, 1, 1, 2), (2, 2, 1, 1), (1, 2, 1, 2)],
                         ids=["x2", "t2", "x2y2", "y2t2"])
def test_faces_reach_their_neighbours(grid):
    world = int(np.prod(grid))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, grid, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        sums = [1.5 * sum(r + 1 for r in range(world)), -2.0 ** -30 * sum(range(world))]
        for r in range(world):
            ok_faces, rc2, v = out[r]
            assert ok_faces, f"rank {r}: a face did not arrive as expected"
            assert rc2 == 0 and v == sums


def test_callback_failure_is_reported():
    """An exception in a callback becomes a non-zero return (DWF_ECOMM in the library)."""
    from paper_1101_0423_gb300 import dwf

    def bad_exchange(send, recv):
        raise RuntimeError("peer lost")

    def bad_allreduce(v):
        raise RuntimeError("peer lost")

    c = dwf.part_comm(bad_exchange, bad_allreduce)
    nb = (ctypes.c_size_t * 8)(*([0] * 8))
    SP = ctypes.c_void_p * 8
    assert c.exchange(None, SP(), SP(), nb) == 1
    v = (ctypes.c_double * 1)(1.0)
    assert c.allreduce(None, v, 1) == 1


def _lonely(rank, world, port, out):
    import time

    import torch.distributed as tdist

    from paper_1101_0423_gb300 import dist as pdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == 0:
            # rank 1 never takes part in the exchange (it failed before the collective step)
            tc = pdist.TorchPartComm((2, 1, 1, 1), pdist.grid_coord(0, (2, 1, 1, 1)), timeout=2.0)
            n = 64
            send = [np.zeros(n, np.uint8) if k < 2 else None for k in range(8)]
            recv = [np.zeros(n, np.uint8) if k < 2 else None for k in range(8)]
            SP = ctypes.c_void_p * 8
            sp = SP(*[x.ctypes.data if x is not None else None for x in send])
            rp = SP(*[x.ctypes.data if x is not None else None for x in recv])
            t0 = time.monotonic()
            rc = tc.comm.exchange(None, sp, rp, (ctypes.c_size_t * 8)(*([n, n] + [0] * 6)))
            out[0] = (rc, time.monotonic() - t0)
        else:
            time.sleep(8.0)
    finally:
        os._exit(0)  # no collective teardown: the peer left mid-protocol


def test_exchange_with_a_failed_peer_times_out():
    """A part whose neighbour failed before the exchange gets a failed callback (DWF_ECOMM in
    the library) after the transport's timeout instead of waiting for ever."""
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_lonely, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
        rc, waited = out[0]
        assert rc == 1 and waited < 7.0
