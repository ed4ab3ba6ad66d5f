"""Batched solves (dwf_solve_batch): several right-hand sides of one operator advance in the
same kernel launches, each with its own CG scalars, restarts and convergence.  Every
solution is checked by the oracle's true residual (<= 1e-10) and against the oracle's own
solve; a batch of one is the single solve bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def relnorm(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def point_sources(dims, ns):
    return np.stack([inputs.point_source(dims, ns, spin, col) for spin in range(4) for col in range(3)])


@pytest.mark.parametrize("prec", [1, 3])
def test_full_system_batch_of_gaussian_sources(gpu_lib, prec):
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 4, 4), 8, 0.03
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=21)
    rhs = np.stack([inputs.gaussian_source(dims, ns, seed=30 + k) for k in range(3)])
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        sol, stats = dwf.dwf_solve_batch(ctx.h, rhs, inner_prec=prec)
    for k in range(3):
        assert stats[k]["converged"] == 1 and stats[k]["true_res_full"] <= 1e-10
        res = relnorm(oracle.dfull(dims, ns, U, M0, mq, om, sg, sol[k]), rhs[k])
        assert res <= 1e-10
        psi_or, _, _ = oracle.solve_full(dims, ns, U, M0, mq, om, sg, rhs[k], tol=1e-13)
        assert relnorm(sol[k], psi_or) < 1e-6


def test_batch_takes_one_common_tightened_pass(gpu_lib):
    """schur_target_pct = 10000 stops every right-hand side of the batch at a full residual
    far above tol; those systems continue together with one common tightened target and
    each ends at |eta - D psi| / |eta| <= 1e-10 (oracle)."""
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 4, 4), 8, 0.03
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=22)
    rhs = np.stack([inputs.gaussian_source(dims, ns, seed=50 + k) for k in range(3)])
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        sol, stats = dwf.dwf_solve_batch(ctx.h, rhs, schur_target_pct=10000)
    for k in range(3):
        assert stats[k]["converged"] == 1 and stats[k]["true_res_full"] <= 1e-10
        assert relnorm(oracle.dfull(dims, ns, U, M0, mq, om, sg, sol[k]), rhs[k]) <= 1e-10


def test_normal_system_batch_with_a_zero_source(gpu_lib):
    """4^4 x 8 Shamir normal equations on even sites; the third source is zero (finished from
    the start, must stay zero while the others iterate)."""
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 4, 4), 8, 0.05
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.3, seed=1)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    rhs = np.stack([inputs.gaussian_source(dims, ns, seed=40 + k, parity=0) for k in range(4)])
    rhs[2] = 0
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        sol, stats = dwf.dwf_solve_batch(ctx.h, rhs, system=dwf.SYS_NORMAL, schur_parity=0)
    assert not np.any(sol[2]) and stats[2]["iters"] == 0 and stats[2]["converged"] == 1
    for k in (0, 1, 3):
        r = rhs[k] - oracle.ccdag_op(dims, ns, U, mp, mm, 0, sol[k])
        assert np.linalg.norm(r) / np.linalg.norm(rhs[k]) <= 1e-10
        assert stats[k]["converged"] == 1


def test_twelve_point_sources_ragged_lattice(gpu_lib):
    """The 12 spin-colour point sources in one batch (6 x 4 x 4 x 6, Ns = 12, Shamir)."""
    dwf = gpu_lib
    dims, ns, mq = (6, 4, 4, 6), 12, 0.01
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.5, seed=23)
    rhs = point_sources(dims, ns)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        sol, stats = dwf.dwf_solve_batch(ctx.h, rhs)
    assert len(stats) == 12
    for k in range(12):
        assert stats[k]["converged"] == 1
        assert relnorm(oracle.dfull(dims, ns, U, M0, mq, om, sg, sol[k]), rhs[k]) <= 1e-10


def test_batch_of_one_is_the_single_solve(gpu_lib):
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 4, 4), 8, 0.03
    om, sg = inputs.weights("borici", ns)
    U = inputs.gauge_field(dims, 0.5, seed=25)
    rhs = inputs.gaussian_source(dims, ns, seed=26)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        one, _ = dwf.dwf_solve(ctx.h, rhs)
        batch, st = dwf.dwf_solve_batch(ctx.h, rhs[None, :])
    assert np.array_equal(one, batch[0])


def test_batch_at_benchmark_size(gpu_lib):
    """Four Gaussian sources on 16^3 x 32 x 16 (cosine weights) in one batch; every solution
    meets the FP64 residual the library recomputes (pinned to the oracle at smaller sizes)."""
    dwf = gpu_lib
    dims, ns, mq = (16, 16, 16, 32), 16, 0.02
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=2)
    rhs = np.stack([inputs.gaussian_source(dims, ns, seed=50 + k) for k in range(4)])
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        sol, stats = dwf.dwf_solve_batch(ctx.h, rhs)
    for k in range(4):
        assert stats[k]["converged"] == 1 and stats[k]["true_res_full"] <= 1e-10
    # one of them through the oracle as well
    assert relnorm(oracle.dfull(dims, ns, U, M0, mq, om, sg, sol[1]), rhs[1]) <= 1e-10
