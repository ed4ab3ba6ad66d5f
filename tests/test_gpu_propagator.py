"""4D quark propagator from 12 point sources solved in one batch (dwf_propagator).

Parity: element by element against the oracle (the same 12 sources solved by the oracle's
Schur solve to 1e-13, the same wall extraction).  Property: for Shamir weights D is
gamma5*R5-hermitian, which makes the wall-projected propagator gamma5-hermitian,
S(x, y)^dagger = g5 S(y, x) g5 -- a check of the source/sink wall convention that fails if
either wall or chirality is swapped.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8
G5 = np.diag([1.0, 1.0, -1.0, -1.0])


def lex(dims, c):
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def oracle_propagator(dims, ns, U, mq, om, sg, x0):
    v4 = int(np.prod(dims))
    prop = np.zeros((v4, 4, 3, 4, 3), complex)
    site0 = lex(dims, x0)
    for beta in range(4):
        for b in range(3):
            src = np.zeros((v4, ns, 4, 3, 2))
            src[site0, 0 if beta < 2 else ns - 1, beta, b, 0] = 1.0
            psi, _, rel = oracle.solve_full(dims, ns, U, M0, mq, om, sg, src.reshape(-1), tol=1e-13)
            psi = psi.view(np.complex128).reshape(v4, ns, 4, 3)
            prop[:, :2, :, beta, b] = psi[:, ns - 1, :2, :]   # P+ from the last slice
            prop[:, 2:, :, beta, b] = psi[:, 0, 2:, :]        # P- from the first slice
    return prop


@pytest.mark.parametrize("kind", ["shamir", "cosine"])
def test_propagator_matches_oracle(gpu_lib, kind):
    dwf = gpu_lib
    dims, ns, mq, x0 = (4, 4, 4, 4), 6, 0.04, (1, 2, 3, 0)
    om, sg = inputs.weights(kind, ns)
    U = inputs.gauge_field(dims, 0.5, seed=31)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        prop, stats = dwf.dwf_propagator(ctx.h, dims, x0)
    assert all(s["converged"] == 1 and s["true_res_full"] <= 1e-10 for s in stats)
    want = oracle_propagator(dims, ns, U, mq, om, sg, x0)
    assert np.max(np.abs(prop - want)) <= 1e-7 * np.max(np.abs(want))


def test_propagator_is_gamma5_hermitian_for_shamir(gpu_lib):
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 2, 6), 8, 0.03
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.5, seed=33)
    x, y = (0, 1, 0, 2), (3, 2, 1, 5)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        px, _ = dwf.dwf_propagator(ctx.h, dims, x)
        py, _ = dwf.dwf_propagator(ctx.h, dims, y)
    s_yx = py[lex(dims, x)].reshape(12, 12)     # S(x <- y): sink x, source y
    s_xy = px[lex(dims, y)].reshape(12, 12)     # S(y <- x)
    g5 = np.kron(G5, np.eye(3))
    lhs = s_yx.conj().T
    rhs = g5 @ s_xy @ g5
    assert np.max(np.abs(lhs - rhs)) <= 1e-8 * np.max(np.abs(rhs))
    # the gamma5 factors matter (the relation is not plain hermiticity)
    assert np.max(np.abs(lhs - s_xy)) > 1e-3 * np.max(np.abs(rhs))
