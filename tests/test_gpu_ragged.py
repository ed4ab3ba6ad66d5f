"""Ragged sets (dwf_solve_ragged): one system on each of several contexts of different Ns,
masses and weights, solved together -- every interval of inner iterations of all of them one
CUDA graph with a branch per context.  Each solution is checked by the oracle's true
residual (<= 1e-10), and against the same context's single solve bit for bit (the same
kernels in the same order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def relnorm(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# (Ns, mq, weights): Ns with the four-site hop layout (multiples of 8) and without (12, 20),
# masses 0.005..0.1 as in the ragged 8-rhs workload
SET = [(8, 0.05, "shamir"), (12, 0.005, "cosine"), (16, 0.02, "borici"), (20, 0.1, "shamir"),
       (24, 0.03, "cosine"), (12, 0.07, "borici")]


def _contexts(dwf, dims, U, members):
    g = dwf.dwf_gauge_create(dims, U)
    try:
        return [dwf.Context(dims, ns, M0, mq, *inputs.weights(w, ns), gauge=g) for ns, mq, w in members]
    finally:
        dwf.dwf_gauge_release(g)


@pytest.mark.parametrize("prec", [1, 3])
def test_ragged_full_system_against_oracle_and_single_solves(gpu_lib, prec):
    dwf = gpu_lib
    dims = (4, 4, 4, 6)
    U = inputs.gauge_field(dims, 0.5, seed=71)
    rhs = [inputs.gaussian_source(dims, ns, seed=300 + k) for k, (ns, _, _) in enumerate(SET)]
    ctxs = _contexts(dwf, dims, U, SET)
    try:
        sol, stats = dwf.dwf_solve_ragged([c.h for c in ctxs], rhs, inner_prec=prec)
        single = [dwf.dwf_solve(c.h, b, inner_prec=prec) for c, b in zip(ctxs, rhs)]
    finally:
        for c in ctxs:
            c.close()
    for k, (ns, mq, w) in enumerate(SET):
        om, sg = inputs.weights(w, ns)
        assert stats[k]["converged"] == 1 and stats[k]["true_res_full"] <= 1e-10
        assert relnorm(oracle.dfull(dims, ns, U, M0, mq, om, sg, sol[k]), rhs[k]) <= 1e-10
        x1, s1 = single[k]
        assert np.array_equal(sol[k], x1)
        assert stats[k]["iters"] == s1["iters"] and stats[k]["restarts"] == s1["restarts"]


def test_ragged_lattices_and_normal_system(gpu_lib):
    """Contexts on two different lattices (their own gauge fields) in one set, normal
    equations on the odd sites; one of the sources is zero."""
    dwf = gpu_lib
    members = [((4, 4, 4, 4), 8, 0.05, "shamir"), ((6, 4, 4, 6), 12, 0.02, "cosine"),
               ((4, 4, 4, 4), 16, 0.03, "borici")]
    ctxs, rhs, fields = [], [], []
    try:
        for k, (dims, ns, mq, w) in enumerate(members):
            U = inputs.gauge_field(dims, 0.4, seed=80 + k)
            om, sg = inputs.weights(w, ns)
            ctxs.append(dwf.Context(dims, ns, M0, mq, om, sg, U))
            b = inputs.gaussian_source(dims, ns, seed=90 + k, parity=1)
            if k == 1:
                b[:] = 0
            rhs.append(b)
            fields.append((dims, ns, mq, om, sg, U))
        sol, stats = dwf.dwf_solve_ragged([c.h for c in ctxs], rhs, system=dwf.SYS_NORMAL, schur_parity=1)
    finally:
        for c in ctxs:
            c.close()
    assert not np.any(sol[1]) and stats[1]["iters"] == 0 and stats[1]["converged"] == 1
    for k in (0, 2):
        dims, ns, mq, om, sg, U = fields[k]
        mp, mm = oracle.m5(ns, M0, mq, om, sg)
        r = rhs[k] - oracle.ccdag_op(dims, ns, U, mp, mm, 1, sol[k])
        assert np.linalg.norm(r) / np.linalg.norm(rhs[k]) <= 1e-10
        assert stats[k]["converged"] == 1


def test_ragged_device_arrays_on_a_stream(gpu_lib):
    """The device form orders the set after the caller's stream and the caller's stream
    after the set: the sources are written on a side stream just before the call, the
    solutions read on it just after."""
    dwf = gpu_lib
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, seed=72)
    members = SET[:3]
    rhs = [inputs.gaussian_source(dims, ns, seed=310 + k) for k, (ns, _, _) in enumerate(members)]
    ctxs = _contexts(dwf, dims, U, members)
    side = torch.cuda.Stream()
    try:
        host = [torch.from_numpy(b).pin_memory() for b in rhs]
        with torch.cuda.stream(side):
            d_rhs = [torch.empty(b.shape, dtype=torch.float64, device="cuda") for b in host]
            d_sol = [torch.empty_like(b) for b in d_rhs]
            for d, h in zip(d_rhs, host):
                d.copy_(h, non_blocking=True)
            stats = dwf.dwf_solve_ragged_dev([c.h for c in ctxs], d_rhs, d_sol, stream=side)
            out = [x.to("cpu", non_blocking=False) for x in d_sol]
        single = [dwf.dwf_solve(c.h, b)[0] for c, b in zip(ctxs, rhs)]
    finally:
        for c in ctxs:
            c.close()
    for k in range(len(members)):
        assert stats[k]["converged"] == 1
        assert np.array_equal(out[k].numpy(), single[k])


def test_ragged_rejects_bad_sets(gpu_lib):
    dwf = gpu_lib
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, seed=73)
    ctxs = _contexts(dwf, dims, U, SET[:2])
    b = [inputs.gaussian_source(dims, ns, seed=1) for ns, _, _ in SET[:2]]
    try:
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_solve_ragged([ctxs[0].h, ctxs[0].h], [b[0], b[0]])
        assert e.value.status == dwf.DWF_EINVAL
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_solve_ragged([c.h for c in ctxs], b, use_x0=1)
        assert e.value.status == dwf.DWF_EINVAL
    finally:
        for c in ctxs:
            c.close()


def test_ragged_member_that_does_not_converge(gpu_lib):
    """A heavy-mass member converges within max_iter (the oracle's FP64 CG on its normal
    equations takes 151 iterations) while a light one does not (404): the set returns
    DWF_ENOCONV, the converged member's solution is its single solve bit for bit (and meets
    the oracle's residual), the other reports converged = 0."""
    dwf = gpu_lib
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, seed=74)
    members = [(8, 0.9, "shamir"), (8, 0.001, "shamir")]
    rhs = [inputs.gaussian_source(dims, ns, seed=320 + k) for k, (ns, _, _) in enumerate(members)]
    ctxs = _contexts(dwf, dims, U, members)
    try:
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_solve_ragged([c.h for c in ctxs], rhs, max_iter=250)
        assert e.value.status == dwf.DWF_ENOCONV
        sol, stats = dwf.dwf_solve_ragged([c.h for c in ctxs], rhs, max_iter=250, allow_noconv=True)
        x0, s0 = dwf.dwf_solve(ctxs[0].h, rhs[0], max_iter=250)
    finally:
        for c in ctxs:
            c.close()
    assert stats[0]["converged"] == 1 and stats[1]["converged"] == 0
    assert stats[0]["iters"] == s0["iters"] and np.array_equal(sol[0], x0)
    om, sg = inputs.weights("shamir", 8)
    assert relnorm(oracle.dfull(dims, 8, U, M0, 0.9, om, sg, sol[0]), rhs[0]) <= 1e-10
