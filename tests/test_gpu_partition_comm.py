"""A domain decomposition across processes: each of two processes holds one part (both on
this one GPU; no kernel waits on another process's kernel -- the faces and sums move
through the host, over gloo), calling dwf_part_apply_comm / dwf_part_solve_comm with the
torch.distributed transport.  The assembled results equal the single-process
decomposition's bit for bit (two parts: the same sums, the same faces) and the oracle's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _blocks(dims, grid, ns):
    """(coord, slices) of every block of a host-layout spinor array shaped (T, Z, Y, X, Ns, 24)."""
    L = [d // g for d, g in zip(dims, grid)]
    out = []
    for r in range(int(np.prod(grid))):
        c, q = [], r
        for g in grid:
            c.append(q % g)
            q //= g
        sl = (slice(c[3] * L[3], (c[3] + 1) * L[3]), slice(c[2] * L[2], (c[2] + 1) * L[2]),
              slice(c[1] * L[1], (c[1] + 1) * L[1]), slice(c[0] * L[0], (c[0] + 1) * L[0]))
        out.append((c, sl))
    return out


def _local(x, dims, ns, sl):
    return np.ascontiguousarray(x.reshape(dims[3], dims[2], dims[1], dims[0], ns, 24)[sl]).reshape(-1)


def _rank(rank, world, port, case, out):
    import torch.distributed as tdist

    from paper_1101_0423_gb300 import dist as pdist, dwf
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, grid, ns, mq, kind, U, x, b, b0, prm, prm16 = case
        om, sg = inputs.weights(kind, ns)
        coord, sl = _blocks(dims, grid, ns)[rank]
        part = dwf.dwf_create_part(dims, grid, coord, ns, M0, mq, om, sg)
        try:
            dwf.dwf_load_gauge_part(part, U)
            tc = pdist.TorchPartComm(grid, coord)
            res = {}
            for op, prec, parity in ((dwf.OP_CCDAG, dwf.PREC_F64, 1), (dwf.OP_C, dwf.PREC_F32, 0),
                                     (dwf.OP_DEO, dwf.PREC_F16, 0)):
                res[(op, prec)] = dwf.dwf_part_apply_comm(part, tc.comm, op, prec, parity, _local(x, dims, ns, sl))
            sol, st = dwf.dwf_part_solve_comm(part, tc.comm, _local(b, dims, ns, sl), **prm)
            res["solve"] = (sol, st["iters"], st["restarts"], st["true_res_full"], st["converged"])
            sol, st = dwf.dwf_part_solve_comm(part, tc.comm, _local(b0, dims, ns, sl), **prm16)
            res["solve16"] = (sol, st["iters"], st["restarts"], st["true_res"], st["converged"])
            out[rank] = res
        finally:
            dwf.dwf_destroy(part)
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("grid", [(2, 1, 1, 1), (1, 1, 1, 2)], ids=["x2", "t2"])
def test_two_processes_one_part_each(gpu_lib, grid):
    dwf = gpu_lib
    dims, ns, mq, kind = (8, 4, 4, 8), 8, 0.05, "cosine"
    U = inputs.gauge_field(dims, 0.5, seed=61)
    x = inputs.gaussian_source(dims, ns, seed=62)
    b = inputs.gaussian_source(dims, ns, seed=63)
    b0 = inputs.gaussian_source(dims, ns, seed=64, parity=0)
    prm = {"inner_prec": dwf.PREC_F32, "tol": 1e-10}
    # normal equations on the even sites with fp16 inner iterations (16-bit faces)
    prm16 = {"inner_prec": dwf.PREC_F16, "tol": 1e-10, "system": dwf.SYS_NORMAL, "schur_parity": 0}
    world = int(np.prod(grid))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        case = (dims, grid, ns, mq, kind, U, x, b, b0, prm, prm16)
        procs = [ctx.Process(target=_rank, args=(r, world, port, case, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = {r: out[r] for r in range(world)}

    def assemble(key):
        g = np.zeros((dims[3], dims[2], dims[1], dims[0], ns, 24))
        for r, (_, sl) in enumerate(_blocks(dims, grid, ns)):
            g[sl] = res[r][key].reshape(g[sl].shape)
        return g.reshape(-1)

    # the same decomposition in this process: both parts here, faces copied on the device
    om, sg = inputs.weights(kind, ns)
    parts = [dwf.dwf_create_part(dims, grid, c, ns, M0, mq, om, sg) for c, _ in _blocks(dims, grid, ns)]
    try:
        for p in parts:
            dwf.dwf_load_gauge_part(p, U)
        mp5, mm5 = oracle.m5(ns, M0, mq, om, sg)
        for op, prec, parity in ((dwf.OP_CCDAG, dwf.PREC_F64, 1), (dwf.OP_C, dwf.PREC_F32, 0),
                                 (dwf.OP_DEO, dwf.PREC_F16, 0)):
            got = assemble((op, prec))
            assert np.array_equal(got, dwf.dwf_part_apply(parts, op, prec, parity, x))
            want = {dwf.OP_CCDAG: lambda: oracle.ccdag_op(dims, ns, U, mp5, mm5, parity, x),
                    dwf.OP_C: lambda: oracle.c_op(dims, ns, U, mp5, mm5, parity, x),
                    dwf.OP_DEO: lambda: oracle.hop(dims, ns, U, 0, x)}[op]()
            tol = {dwf.PREC_F64: 1e-12, dwf.PREC_F32: 1e-5, dwf.PREC_F16: 5e-3}[prec]
            assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol
        sol_1p, st_1p = dwf.dwf_part_solve(parts, b, **prm)
        sol16_1p, st16_1p = dwf.dwf_part_solve(parts, b0, **prm16)
    finally:
        for p in parts:
            dwf.dwf_destroy(p)
    g = np.zeros((dims[3], dims[2], dims[1], dims[0], ns, 24))
    for r, (_, sl) in enumerate(_blocks(dims, grid, ns)):
        g[sl] = res[r]["solve"][0].reshape(g[sl].shape)
    sol = g.reshape(-1)
    for r in range(world):
        _, iters, restarts, rfull, conv = res[r]["solve"]
        assert conv == 1 and iters == st_1p["iters"] and restarts == st_1p["restarts"]
        assert rfull == st_1p["true_res_full"]
    assert np.array_equal(sol, sol_1p)
    r = b - oracle.dfull(dims, ns, U, M0, mq, om, sg, sol)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    g = np.zeros((dims[3], dims[2], dims[1], dims[0], ns, 24))
    for r_, (_, sl) in enumerate(_blocks(dims, grid, ns)):
        g[sl] = res[r_]["solve16"][0].reshape(g[sl].shape)
    sol16 = g.reshape(-1)
    for r_ in range(world):
        _, iters, restarts, rres, conv = res[r_]["solve16"]
        assert conv == 1 and iters == st16_1p["iters"] and restarts == st16_1p["restarts"]
        assert rres == st16_1p["true_res"]
    assert np.array_equal(sol16, sol16_1p)
    r = b0 - oracle.ccdag_op(dims, ns, U, mp5, mm5, 0, sol16)
    assert np.linalg.norm(r) / np.linalg.norm(b0) <= 1e-10
