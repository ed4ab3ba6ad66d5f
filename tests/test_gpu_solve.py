"""GPU solver parity: dwf_solve through the C-ABI against the FP64 CPU oracle.

The binding check of every solve is the true relative residual recomputed by the oracle
from the GPU's solution, |b - C C^dag x| / |b| or |eta - D psi| / |eta| <= 1e-10 (FP64).
The solution is unique, so it must also agree with the oracle's own solve (CG to 1e-13)
within the conditioning bound: |x - x_oracle| / |x_oracle| <= 1e-6 here.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def relnorm(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def config0(gpu_lib):
    """4^4 x Ns=8 Shamir, m0 = 1.8, mq = 0.05, links exp(0.3 i H), Gaussian source on even sites."""
    dims, ns, mq = (4, 4, 4, 4), 8, 0.05
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.3, seed=1)
    b = inputs.gaussian_source(dims, ns, seed=1, parity=0)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    x_or, it, rr = oracle.cg(dims, ns, U, mp, mm, 0, b, tol=1e-13)
    ctx = gpu_lib.Context(dims, ns, M0, mq, om, sg, U)
    yield dict(dims=dims, ns=ns, mq=mq, U=U, b=b, mp=mp, mm=mm, x_or=x_or, ctx=ctx)
    ctx.close()


@pytest.mark.parametrize("prec", [1, 0, 2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_config0_normal_solve(config0, prec, mode):
    from paper_1101_0423_gb300 import dwf
    c = config0
    x, st = dwf.dwf_solve(c["ctx"].h, c["b"], system=dwf.SYS_NORMAL, schur_parity=0, inner_prec=prec,
                          mode=mode, tol=1e-10)
    r = c["b"] - oracle.ccdag_op(c["dims"], c["ns"], c["U"], c["mp"], c["mm"], 0, x)
    res = np.linalg.norm(r) / np.linalg.norm(c["b"])
    assert res <= 1e-10, f"true residual {res:.3e} (stats {st})"
    assert st["converged"] == 1 and st["true_res"] <= 1e-10
    assert abs(st["true_res"] - res) < 1e-11
    assert relnorm(x, c["x_or"]) < 1e-6
    par = inputs.site_parity(c["dims"])
    assert not np.any(x.reshape(len(par), -1)[par == 1])


def test_config0_deterministic_and_graph_invariant(config0):
    from paper_1101_0423_gb300 import dwf
    c = config0
    kw = dict(system=dwf.SYS_NORMAL, schur_parity=0)
    x1, s1 = dwf.dwf_solve(c["ctx"].h, c["b"], use_graph=1, **kw)
    x2, s2 = dwf.dwf_solve(c["ctx"].h, c["b"], use_graph=1, **kw)
    x3, s3 = dwf.dwf_solve(c["ctx"].h, c["b"], use_graph=0, **kw)
    x4, s4 = dwf.dwf_solve(c["ctx"].h, c["b"], use_graph=0, profile=1, **kw)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3) and np.array_equal(x1, x4)
    assert s1["iters"] == s3["iters"] == s4["iters"]
    assert s4["class_launches"]["hop_m5"] == 2 * s4["class_launches"]["hop_update"]


def test_noconv_reports_status(config0):
    from paper_1101_0423_gb300 import dwf
    c = config0
    x, st = dwf.dwf_solve(c["ctx"].h, c["b"], system=dwf.SYS_NORMAL, schur_parity=0, max_iter=5,
                          allow_noconv=True)
    assert st["converged"] == 0 and st["iters"] >= 5
    with pytest.raises(dwf.DwfError) as e:
        dwf.dwf_solve(c["ctx"].h, c["b"], system=dwf.SYS_NORMAL, schur_parity=0, max_iter=5)
    assert e.value.status == dwf.DWF_ENOCONV


def test_zero_source(config0):
    from paper_1101_0423_gb300 import dwf
    c = config0
    x, st = dwf.dwf_solve(c["ctx"].h, np.zeros_like(c["b"]), system=dwf.SYS_NORMAL, schur_parity=0)
    assert not np.any(x) and st["converged"] == 1 and st["iters"] == 0


FULL_CASES = [((4, 4, 4, 4), 8, "cosine", 0.05, 1), ((4, 4, 4, 4), 8, "borici", 0.02, 0),
              ((2, 4, 6, 4), 5, "shamir", 0.1, 1), ((6, 4, 2, 8), 12, "cosine", 0.02, 1),
              ((4, 2, 2, 4), 1, "shamir", 0.05, 1), ((2, 2, 4, 4), 32, "borici", 0.0, 1)]


@pytest.mark.parametrize("dims,ns,kind,mq,sp", FULL_CASES)
@pytest.mark.parametrize("prec", [1, 3])
def test_full_solve_matches_oracle(gpu_lib, dims, ns, kind, mq, sp, prec):
    from paper_1101_0423_gb300 import dwf
    om, sg = inputs.weights(kind, ns)
    U = inputs.gauge_field(dims, 0.5, seed=12)
    eta = inputs.gaussian_source(dims, ns, seed=13)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, schur_parity=sp, inner_prec=prec, tol=1e-10)
    res = np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)) / np.linalg.norm(eta)
    assert res <= 1e-10, f"oracle true residual {res:.3e}, stats {st}"
    assert abs(st["true_res_full"] - res) < 1e-11
    psi_or, _, _ = oracle.solve_full(dims, ns, U, M0, mq, om, sg, eta, p=sp, tol=1e-13)
    assert relnorm(psi, psi_or) < 1e-6


def test_full_size_config1_solve(gpu_lib):
    """16^3 x 32 x Ns=16, cosine weights, mq = 0.02, links exp(0.5 i H): the benchmark's solve,
    FP32 inner CG with FP64 reliable updates; the oracle recomputes |eta - D psi| / |eta|."""
    from paper_1101_0423_gb300 import dwf
    dims, ns, mq = (16, 16, 16, 32), 16, 0.02
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=2)
    eta = inputs.gaussian_source(dims, ns, seed=2)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, tol=1e-10)
    res = np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)) / np.linalg.norm(eta)
    assert res <= 1e-10, f"oracle true residual {res:.3e}, stats {st}"


def test_bf16_inner_escalates_to_fp32_when_its_cycles_fail(gpu_lib):
    """16^3 x 32 x Ns=16 Borici, mq = 0.0064: bf16 inner iterations cannot contract at this
    conditioning; AUTO mode must finish with FP32 inner iterations and meet the residual."""
    from paper_1101_0423_gb300 import dwf
    dims, ns, mq = (16, 16, 16, 32), 16, 0.0064
    om, sg = inputs.weights("borici", ns)
    U = inputs.gauge_field(dims, 0.5, seed=12)
    eta = inputs.gaussian_source(dims, ns, seed=1002)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, inner_prec=dwf.PREC_BF16, tol=1e-10)
    assert st["converged"] == 1 and st["true_res_full"] <= 1e-10
    assert st["escalations"] == 1 and st["inner_prec_used"] == dwf.PREC_F32


@pytest.mark.parametrize("ns", [8, 12])
def test_full_solve_with_optimal_weights(gpu_lib, ns):
    """The optimal domain-wall operator (sigma = omega = the optimal weights for |H_w| in
    [0.05, 6.2], computed by the oracle) solved through the C-ABI; the oracle recomputes
    |eta - D psi| / |eta| and solves the same system."""
    from oracle import weights as OW
    from paper_1101_0423_gb300 import dwf
    dims, mq = (4, 4, 4, 6), 0.02
    om, _ = OW.optimal_weights(ns, 0.05, 6.2)
    U = inputs.gauge_field(dims, 0.5, seed=14)
    eta = inputs.gaussian_source(dims, ns, seed=15)
    with dwf.Context(dims, ns, M0, mq, om, om, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, tol=1e-10)
    res = np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, om, psi)) / np.linalg.norm(eta)
    assert res <= 1e-10 and st["converged"] == 1
    psi_or, _, _ = oracle.solve_full(dims, ns, U, M0, mq, om, om, eta, tol=1e-13)
    assert relnorm(psi, psi_or) < 1e-6


def test_loose_schur_target_takes_the_tightened_pass(gpu_lib):
    """A Schur target of 100 x tol (schur_target_pct = 10000) leaves the full residual of the
    first pass far above tol; the solve must continue from its own x with a tightened target
    and still end at |eta - D psi| / |eta| <= 1e-10 (oracle), with more iterations than a
    solve whose first pass already meets it."""
    from paper_1101_0423_gb300 import dwf
    dims, ns, mq = (4, 4, 4, 6), 8, 0.02
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=16)
    eta = inputs.gaussian_source(dims, ns, seed=17)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, tol=1e-10, schur_target_pct=10000)
        _, st_loose = dwf.dwf_solve(ctx.h, eta, tol=1e-8, schur_target_pct=100)
    res = np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)) / np.linalg.norm(eta)
    assert res <= 1e-10 and st["converged"] == 1 and st["true_res_full"] <= 1e-10
    assert st["iters"] > st_loose["iters"]
