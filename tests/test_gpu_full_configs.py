"""Every workload configuration at its real size, solved on the GPU through the C-ABI, its
true residual recomputed by the FP64 CPU oracle: |eta - D psi| / |eta| <= 1e-10.

- 16^3 x 32 x Ns=16, Borici weights (sigma = omega = 1), mq = 0.02, FP32 inner iterations;
- 16^3 x 32 x Ns=16, cosine weights, mq = 0.02 (the benchmark's inputs), inner iterations in
  FP32, bf16 and fp16 (per-(site, s) norms, 12-real links), each with FP64 restarts;
- 24^3 x 48 x Ns=16 Shamir, mq = 0.01: the 12 spin-colour point sources solved as one batch;
  the oracle recomputes the residual of one source of each chirality wall (each such
  application of D takes the oracle about half a minute on one core), and the library's own
  FP64 residual of all twelve is checked against the same bound.

The solution is unique, so solutions computed with different inner precisions must agree
within the conditioning bound of a 1e-10 residual (checked between FP32 and 16-bit here).
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def oracle_residual(dims, ns, U, mq, om, sg, eta, psi):
    return np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)) / np.linalg.norm(eta)


@pytest.fixture(scope="module")
def lattice16(gpu_lib):
    dims, ns = (16, 16, 16, 32), 16
    U = inputs.gauge_field(dims, 0.5, seed=2)
    eta = inputs.gaussian_source(dims, ns, seed=2)
    return dims, ns, U, eta


def test_config1_borici_full_size(lattice16):
    from paper_1101_0423_gb300 import dwf
    dims, ns, U, eta = lattice16
    mq = 0.02
    om, sg = inputs.weights("borici", ns)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, tol=1e-10)
    res = oracle_residual(dims, ns, U, mq, om, sg, eta, psi)
    assert res <= 1e-10, f"oracle true residual {res:.3e}, stats {st}"
    assert st["converged"] == 1 and abs(st["true_res_full"] - res) < 1e-11


_SWEEP = {}


@pytest.mark.parametrize("prec", [1, 3, 2], ids=["f32", "bf16", "f16"])
def test_config2_precision_sweep_full_size(lattice16, prec):
    from paper_1101_0423_gb300 import dwf
    dims, ns, U, eta = lattice16
    mq = 0.02
    om, sg = inputs.weights("cosine", ns)
    # reliable updates throughout (no switch to defect correction, no escalation to FP32):
    # every inner iteration in the precision under test
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi, st = dwf.dwf_solve(ctx.h, eta, inner_prec=prec, tol=1e-10, mode=dwf.MODE_RELIABLE)
    res = oracle_residual(dims, ns, U, mq, om, sg, eta, psi)
    assert res <= 1e-10, f"oracle true residual {res:.3e}, stats {st}"
    assert st["converged"] == 1
    assert st["escalations"] == 0 and st["inner_prec_used"] == prec and st["mode_used"] == dwf.MODE_RELIABLE
    _SWEEP[prec] = psi
    if prec != 1 and 1 in _SWEEP:
        ref = _SWEEP[1]
        assert np.linalg.norm(psi - ref) / np.linalg.norm(ref) < 1e-6


def test_config3_point_sources_24x48_full_size(gpu_lib):
    import torch
    from paper_1101_0423_gb300 import dwf
    dims, ns, mq = (24, 24, 24, 48), 16, 0.01
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.5, seed=3)
    src = [(spin, col) for spin in range(4) for col in range(3)]
    d_rhs = torch.from_numpy(np.stack([inputs.point_source(dims, ns, s, c) for s, c in src])).cuda()
    d_sol = torch.empty_like(d_rhs)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        stream = torch.cuda.current_stream()
        stats = dwf.dwf_solve_batch_dev(ctx.h, 12, d_rhs, d_sol, stream=stream)
        stream.synchronize()
    assert all(s["converged"] == 1 and s["true_res_full"] <= 1e-10 for s in stats)
    for k in (0, 11):  # spin 0 colour 0 (wall s = 0) and spin 3 colour 2 (wall s = Ns - 1)
        eta = d_rhs[k].cpu().numpy()
        psi = d_sol[k].cpu().numpy()
        res = oracle_residual(dims, ns, U, mq, om, sg, eta, psi)
        assert res <= 1e-10, f"source {src[k]}: oracle true residual {res:.3e}, stats {stats[k]}"
        assert abs(stats[k]["true_res_full"] - res) < 1e-11
