"""Warm start (use_x0): Algorithm 2 started from a given x_hat.  The solve from an initial
guess must meet the same oracle-recomputed residual as a cold solve, relative to the
original right-hand side, need fewer inner iterations from a close guess, stop at once when
the guess already meets the tolerance, and ignore whatever the guess holds where the
system has no unknowns."""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def relres_full(case, psi, eta):
    d = case
    return np.linalg.norm(eta - oracle.dfull(d["dims"], d["ns"], d["U"], M0, d["mq"], d["om"], d["sg"], psi)) \
        / np.linalg.norm(eta)


@pytest.fixture(scope="module")
def case(gpu_lib):
    dims, ns, mq = (4, 4, 4, 6), 8, 0.02
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=131)
    ctx = gpu_lib.Context(dims, ns, M0, mq, om, sg, U)
    eta = inputs.gaussian_source(dims, ns, seed=132)
    yield dict(dims=dims, ns=ns, mq=mq, om=om, sg=sg, U=U, ctx=ctx, eta=eta)
    ctx.close()


def test_full_system_from_a_close_guess(gpu_lib, case):
    dwf = gpu_lib
    eta = case["eta"]
    psi_cold, st_cold = dwf.dwf_solve(case["ctx"].h, eta)
    rng = np.random.default_rng(133)
    x0 = psi_cold * (1 + 1e-5 * rng.standard_normal(psi_cold.shape))
    psi, st = dwf.dwf_solve(case["ctx"].h, eta, x0=x0)
    res = relres_full(case, psi, eta)
    assert st["converged"] == 1 and res <= 1e-10
    assert abs(st["true_res_full"] - res) < 1e-11
    assert 0 < st["iters"] < st_cold["iters"]


def test_guess_that_already_meets_tol_returns_it(gpu_lib, case):
    dwf = gpu_lib
    eta = case["eta"]
    psi_or, _, _ = oracle.solve_full(case["dims"], case["ns"], case["U"], M0, case["mq"], case["om"], case["sg"],
                                     eta, tol=1e-13)
    psi, st = dwf.dwf_solve(case["ctx"].h, eta, x0=psi_or)
    assert st["converged"] == 1 and st["iters"] == 0 and st["true_res_full"] <= 1e-10
    assert np.array_equal(psi, psi_or)


def test_zero_source_returns_zero_whatever_the_guess(gpu_lib, case):
    dwf = gpu_lib
    x0 = inputs.gaussian_source(case["dims"], case["ns"], seed=134)
    psi, st = dwf.dwf_solve(case["ctx"].h, np.zeros_like(x0), x0=x0)
    assert st["converged"] == 1 and not np.any(psi)


def test_normal_system_ignores_the_other_parity_of_the_guess(gpu_lib, case):
    """C C^dag x = b on even sites from a guess that also has odd-site entries: the odd
    sites come back as 0 and the even sites solve the system (oracle residual)."""
    dwf = gpu_lib
    d = case
    mp, mm = oracle.m5(d["ns"], M0, d["mq"], d["om"], d["sg"])
    b = inputs.gaussian_source(d["dims"], d["ns"], seed=135, parity=0)
    x_cold, st_cold = dwf.dwf_solve(d["ctx"].h, b, system=dwf.SYS_NORMAL, schur_parity=0)
    noise = inputs.gaussian_source(d["dims"], d["ns"], seed=136)
    x0 = x_cold + 1e-6 * noise  # noise on both parities
    x, st = dwf.dwf_solve(d["ctx"].h, b, x0=x0, system=dwf.SYS_NORMAL, schur_parity=0)
    par = np.repeat(inputs.site_parity(d["dims"]), d["ns"] * 24)
    assert not np.any(x[par == 1])
    r = b - oracle.ccdag_op(d["dims"], d["ns"], d["U"], mp, mm, 0, x)
    res = np.linalg.norm(r) / np.linalg.norm(b)
    assert st["converged"] == 1 and res <= 1e-10 and abs(st["true_res"] - res) < 1e-11
    assert st["iters"] < st_cold["iters"]


def test_batch_with_guesses(gpu_lib, case):
    dwf = gpu_lib
    d = case
    rhs = np.stack([inputs.gaussian_source(d["dims"], d["ns"], seed=140 + k) for k in range(2)])
    x0 = np.stack([np.zeros_like(rhs[0]), 0.5 * inputs.gaussian_source(d["dims"], d["ns"], seed=150)])
    sol, stats = dwf.dwf_solve_batch(d["ctx"].h, rhs, x0=x0)
    for k in range(2):
        assert stats[k]["converged"] == 1 and relres_full(case, sol[k], rhs[k]) <= 1e-10
