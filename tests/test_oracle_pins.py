"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the Clifford
algebra, the free-field momentum form of D_w, gamma5- and gamma5*R5-hermiticity,
gauge covariance, the closed form of the Shamir M5, the identity of the two forms
of M5 in Eq. 8, a brute-force dense assembly with an LU solve, and the Schur
solve against the unpreconditioned solve.  A dropped term, a wrong sign or index,
or a transposed operand anywhere in the oracle fails at least one of them.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs
from tests import dense

M0 = 1.8


def cview(a, dims, ns):
    return a.view(np.complex128).reshape(int(np.prod(dims)), ns, 4, 3)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------ gamma basis

def test_gamma_clifford_and_gamma5():
    g = [oracle.gamma(mu) for mu in range(4)]
    g5 = oracle.gamma(4)
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)          # Hermitian
        assert np.allclose(g5 @ g[a] + g[a] @ g5, 0, atol=0)     # anticommutes with gamma_5
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4), atol=0)
    # chiral basis: P+ = (1+g5)/2 selects spins 0,1 (the reading used for Eq. 3)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    gd, gd5 = dense.gammas()
    for a in range(4):
        assert np.allclose(g[a], gd[a], atol=0)


# ------------------------------------------------------------------ D_w (Eq. 2)

@pytest.mark.parametrize("dims", [(4, 6, 2, 8), (2, 4, 6, 4)])
def test_free_field_momentum_closed_form(dims):
    """U = 1: D_w e^{ipx} chi = [(4 - m0) - sum cos p + i sum gamma_mu sin p] e^{ipx} chi."""
    ns = 2
    V = int(np.prod(dims))
    U = inputs.unit_gauge(dims)
    g = dense.gammas()[0]
    coords = np.array(dense.coords(dims))
    rng = np.random.default_rng(7)
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 2, 1, 3)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        chi = rng.normal(size=(ns, 4, 3)) + 1j * rng.normal(size=(ns, 4, 3))
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None, None, None] * chi[None]
        out = cview(oracle.dw(dims, ns, U, M0, psi.view(np.float64).reshape(-1)), dims, ns)
        Dp = (4 - M0 - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        want = phase[:, None, None, None] * np.einsum("ab,sbc->sac", Dp, chi)[None]
        assert rel(out, want) < 1e-13


def eq4_l(ns, mq):
    """L+ and L- of Eq. 3-4 (0-based s): (L+)_{s,s-1} = 1, corner (L+)_{0,Ns-1} = -mq/(2 m0)."""
    Lp = np.zeros((ns, ns))
    for s in range(1, ns):
        Lp[s, s - 1] = 1.0
    Lp[0, ns - 1] = -mq / (2 * M0)
    return Lp, Lp.T


@pytest.mark.parametrize("dims,ns", [((4, 6, 2, 8), 4), ((2, 4, 6, 4), 3)])
def test_free_5d_operator_momentum_block(dims, ns):
    """U = 1: D of Eq. 1 maps e^{ipx} chi to e^{ipx} D(p) chi with the 4Ns x 4Ns (per colour)
    block D(p) chi = D_w(p) [(omega + sigma L) chi] + (1 - L) chi, where D_w(p) is the free
    Wilson matrix of the momentum and L = P+ L+ + P- L- acts along s (Eq. 3-4).  Distinct
    random omega and sigma, so no weight can stand in for the other."""
    mq = 0.07
    U = inputs.unit_gauge(dims)
    g = dense.gammas()[0]
    coords = np.array(dense.coords(dims))
    rng = np.random.default_rng(17)
    om, sg = rng.uniform(0.5, 1.5, ns), rng.uniform(-0.4, 0.9, ns)
    Lp, Lm = eq4_l(ns, mq)
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 2, 0, 1), (1, 1, 1, 3)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        chi = rng.normal(size=(ns, 4, 3)) + 1j * rng.normal(size=(ns, 4, 3))
        phase = np.exp(1j * coords @ p)
        psi = phase[:, None, None, None] * chi[None]
        out = cview(oracle.dfull(dims, ns, U, M0, mq, om, sg, psi.view(np.float64).reshape(-1)), dims, ns)
        Lchi = np.concatenate([np.einsum("st,tac->sac", Lp, chi[:, :2]), np.einsum("st,tac->sac", Lm, chi[:, 2:])],
                              axis=1)
        chi1 = om[:, None, None] * chi + sg[:, None, None] * Lchi
        Dp = (4 - M0 - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        block = np.einsum("ab,sbc->sac", Dp, chi1) + chi - Lchi
        assert rel(out, phase[:, None, None, None] * block[None]) < 1e-13


@pytest.mark.parametrize("p_sch", [0, 1])
def test_free_field_solve_is_the_inverse_momentum_block(p_sch):
    """U = 1, eta = e^{ipx} chi: the even-odd solve of Eq. 10 (source preparation, CG on
    C C^dag, reconstruction) must return e^{ipx} D(p)^{-1} chi, with D(p) the 4Ns x 4Ns
    momentum block of Eq. 1 (per colour), inverted here with numpy."""
    dims, ns, mq = (4, 2, 2, 4), 4, 0.05
    U = inputs.unit_gauge(dims)
    g = dense.gammas()[0]
    coords = np.array(dense.coords(dims))
    rng = np.random.default_rng(19)
    om, sg = rng.uniform(0.6, 1.4, ns), rng.uniform(-0.3, 0.8, ns)
    Lp, Lm = eq4_l(ns, mq)
    P = [np.diag([1, 1, 0, 0]).astype(complex), np.diag([0, 0, 1, 1]).astype(complex)]
    Lfull = np.kron(Lp, P[0]) + np.kron(Lm, P[1])          # (s, spin) x (s', spin')
    W = np.kron(np.diag(om), np.eye(4)) + np.diag(np.repeat(sg, 4)) @ Lfull
    for n in [(1, 0, 0, 1), (0, 1, 1, 3)]:
        p = 2 * np.pi * np.array(n) / np.array(dims)
        Dp = (4 - M0 - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        block = np.kron(np.eye(ns), Dp) @ W + np.eye(4 * ns) - Lfull
        chi = rng.normal(size=(ns, 4, 3)) + 1j * rng.normal(size=(ns, 4, 3))
        phase = np.exp(1j * coords @ p)
        eta = (phase[:, None, None, None] * chi[None]).view(np.float64).reshape(-1)
        psi, _, relres = oracle.solve_full(dims, ns, U, M0, mq, om, sg, eta, p=p_sch, tol=1e-13)
        want = np.linalg.solve(block, chi.reshape(4 * ns, 3)).reshape(ns, 4, 3)
        assert relres < 1e-12
        assert rel(cview(psi, dims, ns), phase[:, None, None, None] * want[None]) < 1e-10


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_gamma5_hermiticity_of_dw(dims):
    """<chi, g5 D_w g5 psi> = <D_w chi, psi> for a random gauge field."""
    ns = 2
    U = inputs.gauge_field(dims, 0.5, seed=11)
    psi = inputs.gaussian_source(dims, ns, seed=12)
    chi = inputs.gaussian_source(dims, ns, seed=13)

    def g5(v):
        c = cview(v.copy(), dims, ns)
        c[:, :, 2:, :] *= -1
        return c.view(np.float64).reshape(-1)

    lhs = oracle.dot(chi, g5(oracle.dw(dims, ns, U, M0, g5(psi))))
    rhs = oracle.dot(oracle.dw(dims, ns, U, M0, chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_gauge_covariance(dims):
    """D[U^W] (W psi) = W D[U] psi with U^W_mu(x) = W(x) U_mu(x) W(x+mu)^dag."""
    ns = 2
    V = int(np.prod(dims))
    U = inputs.gauge_field(dims, 0.5, seed=21)
    W = inputs.gauge_transform(dims, seed=22)
    Uc = U.view(np.complex128).reshape(V, 4, 3, 3)
    UW = np.empty_like(Uc)
    for site, c in enumerate(dense.coords(dims)):
        for mu in range(4):
            cf = list(c)
            cf[mu] = (cf[mu] + 1) % dims[mu]
            UW[site, mu] = W[site] @ Uc[site, mu] @ W[dense.lex(dims, cf)].conj().T
    psi = inputs.gaussian_source(dims, ns, seed=23)
    rot = lambda v: np.einsum("xab,xsib->xsia", W, cview(v, dims, ns)).reshape(-1).view(np.float64)
    lhs = oracle.dw(dims, ns, UW.view(np.float64).reshape(-1), M0, rot(psi))
    rhs = rot(oracle.dw(dims, ns, U, M0, psi))
    assert rel(lhs, rhs) < 1e-13


def test_hop_blocks_are_the_offdiagonal_part_of_dw():
    """Eq. 12 blocks: D_w = (4 - m0) + D^{EO} + D^{OE} (Eq. 6 block form)."""
    dims, ns = (4, 2, 2, 4), 3
    U = inputs.gauge_field(dims, 0.5, seed=31)
    psi = inputs.gaussian_source(dims, ns, seed=32)
    full = oracle.dw(dims, ns, U, M0, psi)
    split = (4 - M0) * psi + oracle.hop(dims, ns, U, 0, psi) + oracle.hop(dims, ns, U, 1, psi)
    assert rel(split, full) < 1e-14
    # D^{p,1-p} reads only parity 1-p and writes only parity p
    par = inputs.site_parity(dims)
    for p in (0, 1):
        h = cview(oracle.hop(dims, ns, U, p, psi), dims, ns)
        assert np.all(h[par != p] == 0)
        masked = cview(psi.copy(), dims, ns)
        masked[par == p] = 0
        h2 = oracle.hop(dims, ns, U, p, masked.view(np.float64).reshape(-1))
        assert np.array_equal(h.view(np.float64).reshape(-1), h2)


@pytest.mark.parametrize("p", [0, 1])
def test_hop_dag_is_the_adjoint(p):
    dims, ns = (2, 4, 6, 4), 3
    U = inputs.gauge_field(dims, 0.5, seed=41)
    par = inputs.site_parity(dims)
    a = cview(inputs.gaussian_source(dims, ns, seed=42), dims, ns)
    b = cview(inputs.gaussian_source(dims, ns, seed=43), dims, ns)
    a[par == p] = 0          # input of D^{p,1-p}
    b[par != p] = 0          # output side
    a, b = a.view(np.float64).reshape(-1), b.view(np.float64).reshape(-1)
    lhs = oracle.dot(b, oracle.hop(dims, ns, U, p, a))
    rhs = oracle.dot(oracle.hop_dag(dims, ns, U, p, b), a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ------------------------------------------------------------------ fifth dimension

@pytest.mark.parametrize("ns,mq", [(4, 0.05), (5, 0.02), (8, 0.1), (16, 0.01)])
def test_m5_shamir_closed_form(ns, mq):
    """Shamir (sigma = 0, omega = 1): M5 = (a - L+)^{-1}, a = 5 - m0, summed as a geometric series:
    (M5+)_{ss'} = a^{-1-k} / (1 - kappa a^{-Ns}) * (kappa if s < s' else 1), k = (s - s') mod Ns,
    kappa = -mq/(2 m0).  M5- is its transpose."""
    om, sg = inputs.weights("shamir", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    a, kappa = 5.0 - M0, -mq / (2 * M0)
    want = np.zeros((ns, ns))
    for s in range(ns):
        for t in range(ns):
            k = (s - t) % ns
            want[s, t] = a ** (-1 - k) / (1 - kappa * a ** (-ns)) * (kappa if s < t else 1.0)
    assert np.max(np.abs(mp - want)) < 1e-15
    assert np.max(np.abs(mm - want.T)) < 1e-15


@pytest.mark.parametrize("ns", [3, 4, 8, 16])
@pytest.mark.parametrize("mq", [0.05, 0.4])
def test_m5_borici_spectrum(ns, mq):
    """Borici (sigma = omega = 1, so c = 1): Eq. 8 reads M5 = [(4 - m0) + (1 - L)(1 + L)^{-1}]^{-1}.
    L+ shifts s up by one and wraps with the factor kappa = -mq/(2 m0) (Eq. 4), so
    L+^Ns = kappa and its eigenvalues are the Ns roots lam of lam^Ns = kappa; M5+ then has
    the eigenvalues 1 / [(4 - m0) + (1 - lam)/(1 + lam)], and M5- = M5+^T the same."""
    om, sg = inputs.weights("borici", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    kappa = -mq / (2 * M0)
    lam = abs(kappa) ** (1.0 / ns) * np.exp(1j * np.pi * (2 * np.arange(ns) + 1) / ns)  # kappa < 0
    want = 1.0 / ((4 - M0) + (1 - lam) / (1 + lam))
    for m in (mp, mm):
        got = np.linalg.eigvals(m)
        # match each predicted eigenvalue to the nearest computed one (a permutation)
        d = np.abs(got[:, None] - want[None, :])
        assert np.all(np.sort(d.min(axis=0)) < 1e-12)
        assert sorted(np.argmin(d, axis=0)) == list(range(ns))


def test_lmat_is_eq4():
    lp, lm = oracle.lmat(5, M0, 0.07)
    want = np.zeros((5, 5))
    want[0, 4] = -0.07 / (2 * M0)
    for s in range(1, 5):
        want[s, s - 1] = 1
    assert np.array_equal(lp, want) and np.array_equal(lm, want.T)


@pytest.mark.parametrize("kind", ["shamir", "borici", "cosine", "mixed"])
def test_m5_two_forms_of_eq8(kind):
    """M5 = omega^{-1/2} Y X^{-1} omega^{1/2} (first form, from X and Y of Eq. 7) equals the
    oracle's second form; S1 and S2 of Eq. 9 follow from the same X, Y."""
    ns, mq = 8, 0.03
    if kind == "mixed":
        om = 1.0 + 0.3 * np.sin(np.arange(ns) + 0.4)
        sg = 0.5 + 0.2 * np.cos(np.arange(ns))
    else:
        om, sg = inputs.weights(kind, ns)
    lp, lm = dense.lmats(ns, M0, mq)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    s1p, s1m, s2p, s2m = oracle.s1s2(ns, M0, mq, om, sg)
    for L, m5o, s1o, s2o in ((lp, mp, s1p, s2p), (lm, mm, s1m, s2m)):
        c = np.diag(sg / om)
        Y = np.diag(om) @ (np.eye(ns) + c @ L)
        X = (4 - M0) * Y + (np.eye(ns) - L)
        rw = np.diag(np.sqrt(om))
        M5 = np.linalg.inv(rw) @ Y @ np.linalg.inv(X) @ rw
        assert np.max(np.abs(m5o - M5)) < 1e-13
        assert np.max(np.abs(s1o - np.linalg.inv(rw) @ Y @ np.linalg.inv(X))) < 1e-13
        assert np.max(np.abs(s2o - np.linalg.inv(Y) @ rw)) < 1e-13
    if kind != "mixed":          # constant c = sigma/omega: M5- = M5+^T
        assert np.max(np.abs(mm - mp.T)) < 1e-14


# ------------------------------------------------------------------ Eq. 1 / Eq. 5: dense assembly

CASES = [((2, 2, 2, 2), 4, "shamir"), ((2, 2, 2, 4), 3, "cosine"), ((4, 2, 2, 2), 3, "borici"),
         ((2, 2, 2, 2), 4, "cosine")]


@pytest.mark.parametrize("dims,ns,kind", CASES)
def test_dfull_matches_dense_assembly(dims, ns, kind):
    mq = 0.05
    U = inputs.gauge_field(dims, 0.5, seed=51)
    om, sg = inputs.weights(kind, ns)
    D = dense.dense_d5(dims, ns, U, M0, mq, om, sg)
    psi = inputs.gaussian_source(dims, ns, seed=52)
    out = oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)
    want = (D @ psi.view(np.complex128)).view(np.float64)
    assert rel(out, want) < 1e-13


@pytest.mark.parametrize("dims,ns,kind", CASES)
@pytest.mark.parametrize("p", [0, 1])
def test_schur_solve_matches_dense_lu(dims, ns, kind, p):
    """The even-odd Schur path of Eq. 10-11 + CG gives the unpreconditioned LU solution."""
    mq = 0.05
    U = inputs.gauge_field(dims, 0.5, seed=61)
    om, sg = inputs.weights(kind, ns)
    D = dense.dense_d5(dims, ns, U, M0, mq, om, sg)
    eta = inputs.gaussian_source(dims, ns, seed=62)
    psi, iters, relres = oracle.solve_full(dims, ns, U, M0, mq, om, sg, eta, p=p, tol=1e-14)
    want = np.linalg.solve(D, eta.view(np.complex128)).view(np.float64)
    assert relres < 1e-13
    assert rel(psi, want) < 1e-11


def test_ldu_factorisation_of_eq10():
    """D = S1^{-1} [[1, M5 D^EO], [M5 D^OE, 1]] S2^{-1}: apply the right side to a vector."""
    dims, ns, mq = (2, 2, 2, 4), 4, 0.04
    U = inputs.gauge_field(dims, 0.5, seed=71)
    om, sg = inputs.weights("cosine", ns)
    psi = inputs.gaussian_source(dims, ns, seed=72)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    s1p, s1m, s2p, s2m = oracle.s1s2(ns, M0, mq, om, sg)
    inv = np.linalg.inv
    # S2^{-1} psi
    a = oracle.apply_s(dims, ns, inv(s2p), inv(s2m), psi)
    # [[1, M5 D^{EO}], [M5 D^{OE}, 1]] a  =  a + M5 (D^{EO} + D^{OE}) a
    h = oracle.hop(dims, ns, U, 0, a) + oracle.hop(dims, ns, U, 1, a)
    b = a + oracle.apply_s(dims, ns, mp, mm, h)
    out = oracle.apply_s(dims, ns, inv(s1p), inv(s1m), b)
    want = oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)
    assert rel(out, want) < 1e-13


# ------------------------------------------------------------------ hermiticity of D (gamma5 R5)

def _g5r5(v, dims, ns):
    c = cview(v.copy(), dims, ns)[:, ::-1].copy()
    c[:, :, 2:, :] *= -1
    return c.view(np.float64).reshape(-1)


def test_gamma5_r5_hermiticity_shamir():
    """Shamir: Gamma D Gamma = D^dagger with Gamma = gamma5 R5 (R5: s -> Ns-1-s)."""
    dims, ns, mq = (2, 4, 2, 4), 6, 0.05
    U = inputs.gauge_field(dims, 0.5, seed=81)
    om, sg = inputs.weights("shamir", ns)
    psi = inputs.gaussian_source(dims, ns, seed=82)
    chi = inputs.gaussian_source(dims, ns, seed=83)
    D = lambda v: oracle.dfull(dims, ns, U, M0, mq, om, sg, v)
    lhs = oracle.dot(chi, _g5r5(D(_g5r5(psi, dims, ns)), dims, ns))
    rhs = oracle.dot(D(chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


@pytest.mark.parametrize("kind", ["borici", "symmetric"])
def test_gamma5_r5_hermiticity_of_d_times_inverse_one_plus_cl(kind):
    """sigma = omega with R5-symmetric omega: Gamma D (1+cL)^{-1} Gamma = (D (1+cL)^{-1})^dagger."""
    dims, ns, mq = (2, 4, 2, 4), 6, 0.05
    U = inputs.gauge_field(dims, 0.5, seed=91)
    om, sg = inputs.weights(kind, ns)
    assert np.allclose(om, om[::-1])
    lp, lm = dense.lmats(ns, M0, mq)
    c = np.diag(sg / om)
    ip, im = np.linalg.inv(np.eye(ns) + c @ lp), np.linalg.inv(np.eye(ns) + c @ lm)
    psi = inputs.gaussian_source(dims, ns, seed=92)
    chi = inputs.gaussian_source(dims, ns, seed=93)
    K = lambda v: oracle.dfull(dims, ns, U, M0, mq, om, sg, oracle.apply_s(dims, ns, ip, im, v))
    lhs = oracle.dot(chi, _g5r5(K(_g5r5(psi, dims, ns)), dims, ns))
    rhs = oracle.dot(K(chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_gamma5_r5_fails_for_cosine_weights():
    """The cosine weights are not R5-symmetric, so the identity above must NOT hold (guards
    against a test that passes for any operator)."""
    dims, ns, mq = (2, 4, 2, 4), 6, 0.05
    U = inputs.gauge_field(dims, 0.5, seed=91)
    om, sg = inputs.weights("cosine", ns)
    lp, lm = dense.lmats(ns, M0, mq)
    ip, im = np.linalg.inv(np.eye(ns) + lp), np.linalg.inv(np.eye(ns) + lm)
    psi = inputs.gaussian_source(dims, ns, seed=92)
    chi = inputs.gaussian_source(dims, ns, seed=93)
    K = lambda v: oracle.dfull(dims, ns, U, M0, mq, om, sg, oracle.apply_s(dims, ns, ip, im, v))
    lhs = oracle.dot(chi, _g5r5(K(_g5r5(psi, dims, ns)), dims, ns))
    rhs = oracle.dot(K(chi), psi)
    assert abs(lhs - rhs) > 1e-3 * abs(rhs)


# ------------------------------------------------------------------ C, C^dagger, CG

@pytest.mark.parametrize("p", [0, 1])
def test_cdag_is_adjoint_and_gamma5_identity(p):
    """or_cdag is the adjoint of or_c, and equals g5 (1 - D^{p,1-p} M5^T D^{1-p,p} M5^T) g5."""
    dims, ns, mq = (2, 4, 2, 4), 4, 0.05
    U = inputs.gauge_field(dims, 0.5, seed=101)
    om, sg = inputs.weights("cosine", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    par = inputs.site_parity(dims)

    def on_p(seed):
        v = cview(inputs.gaussian_source(dims, ns, seed=seed), dims, ns)
        v[par != p] = 0
        return v.view(np.float64).reshape(-1)

    a, b = on_p(102), on_p(103)
    lhs = oracle.dot(b, oracle.c_op(dims, ns, U, mp, mm, p, a))
    rhs = oracle.dot(oracle.cdag_op(dims, ns, U, mp, mm, p, b), a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)

    def g5(v):
        c = cview(v.copy(), dims, ns)
        c[:, :, 2:, :] *= -1
        return c.view(np.float64).reshape(-1)

    t = oracle.apply_s(dims, ns, mp, mm, g5(a), transpose=True, parity=p)
    t = oracle.hop(dims, ns, U, 1 - p, t)
    t = oracle.apply_s(dims, ns, mp, mm, t, transpose=True, parity=1 - p)
    t = oracle.hop(dims, ns, U, p, t)
    want = g5(g5(a) - t)
    assert rel(oracle.cdag_op(dims, ns, U, mp, mm, p, a), want) < 1e-13


def test_ccdag_hermitian_positive_definite():
    dims, ns, mq, p = (2, 2, 2, 2), 2, 0.05, 1
    U = inputs.gauge_field(dims, 0.5, seed=111)
    om, sg = inputs.weights("cosine", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    par = inputs.site_parity(dims)
    V = int(np.prod(dims))
    idx = [i for i in range(V * ns * 12) if par[i // (ns * 12)] == p]
    A = np.zeros((len(idx), len(idx)), complex)
    for j, col in enumerate(idx):
        e = np.zeros(V * ns * 12, complex)
        e[col] = 1
        out = oracle.ccdag_op(dims, ns, U, mp, mm, p, e.view(np.float64)).view(np.complex128)
        A[:, j] = out[idx]
    assert np.max(np.abs(A - A.conj().T)) < 1e-14 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0


def test_cg_reaches_tolerance_config0_size():
    """4^4 x Ns=8 Shamir, mq = 0.05, source on even sites, CG on C C^dag (even Schur parity)."""
    dims, ns, mq = (4, 4, 4, 4), 8, 0.05
    U = inputs.gauge_field(dims, 0.3, seed=1)
    om, sg = inputs.weights("shamir", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    b = inputs.gaussian_source(dims, ns, seed=1, parity=0)
    x, iters, relres = oracle.cg(dims, ns, U, mp, mm, 0, b, tol=1e-12)
    assert relres < 1e-12 and 0 < iters < 2000
    # residual recomputed outside the CG routine
    r = b - oracle.ccdag_op(dims, ns, U, mp, mm, 0, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-12


@pytest.mark.parametrize("k", [3, 7])
def test_cg_iterates_are_the_krylov_galerkin_solutions(k):
    """Algorithm 1 from x0 = 0 stopped after k iterations gives the x in the Krylov space
    K_k = span{b, Ab, ..., A^{k-1} b} whose residual is orthogonal to K_k (A = C C^dag
    Hermitian positive definite): the defining property of CG, which holds only if every
    alpha and beta is right and the search directions are A-conjugate.  The Galerkin solution
    is formed here from an orthonormal basis of K_k and a k x k solve."""
    dims, ns, mq, p = (4, 4, 4, 4), 4, 0.05, 1
    U = inputs.gauge_field(dims, 0.5, seed=121)
    om, sg = inputs.weights("cosine", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    b = inputs.gaussian_source(dims, ns, seed=122, parity=p)
    A = lambda v: oracle.ccdag_op(dims, ns, U, mp, mm, p, np.ascontiguousarray(v).view(np.float64)).view(np.complex128)
    bc = b.view(np.complex128)
    Q = np.zeros((bc.size, k), complex)
    v = bc.copy()
    for j in range(k):  # Arnoldi with Gram-Schmidt applied twice
        for _ in range(2):
            v = v - Q[:, :j] @ (Q[:, :j].conj().T @ v)
        Q[:, j] = v / np.linalg.norm(v)
        v = A(Q[:, j])
    AQ = np.stack([A(Q[:, j]) for j in range(k)], axis=1)
    y = np.linalg.solve(Q.conj().T @ AQ, Q.conj().T @ bc)
    x_gal = Q @ y
    x, iters, _ = oracle.cg(dims, ns, U, mp, mm, p, b, tol=1e-300, maxiter=k)
    assert iters == k
    xc = x.view(np.complex128)
    assert np.linalg.norm(xc - x_gal) / np.linalg.norm(x_gal) < 1e-10
    r = bc - A(xc)
    assert np.linalg.norm(Q.conj().T @ r) < 1e-10 * np.linalg.norm(r)


def test_cg_error_decreases_monotonically_in_the_a_norm():
    """A CG invariant: the A-norm of the error |x_k - x*|_A (A = C C^dag) falls strictly with
    every iteration (x* from a solve to 1e-13)."""
    dims, ns, mq, p = (2, 4, 2, 4), 4, 0.05, 0
    U = inputs.gauge_field(dims, 0.5, seed=141)
    om, sg = inputs.weights("borici", ns)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    b = inputs.gaussian_source(dims, ns, seed=142, parity=p)
    xs, _, rr = oracle.cg(dims, ns, U, mp, mm, p, b, tol=1e-13, maxiter=3000)
    assert rr < 1e-13
    prev = np.inf
    for k in range(1, 16):
        x, iters, _ = oracle.cg(dims, ns, U, mp, mm, p, b, tol=1e-300, maxiter=k)
        e = x - xs
        ea = np.sqrt(oracle.dot(e, oracle.ccdag_op(dims, ns, U, mp, mm, p, e)).real)
        assert iters == k and ea < prev
        prev = ea
