"""Brute-force dense assembly of the domain-wall operator for tiny lattices (tests only).

Built from the definitions with numpy, independently of the oracle's C loops:
  D_w   Eq. 2 (4D Wilson operator with the (d - m0) term, d = 4), as a dense
        (12 V4) x (12 V4) matrix indexed (site, spin, colour);
  L     Eq. 3-4, L = P+ (x) L+ + P- (x) L-;
  D     Eq. 5, D = D_w (omega + sigma L) + (1 - L), indexed (site, s, spin, colour)
        like the host layout of Sec. 3.1.
The gamma basis is the chiral one (gamma_k = [[0, -i s_k], [i s_k, 0]],
gamma_4 = [[0, 1], [1, 0]]), written out again here rather than taken from the oracle.
"""
import numpy as np

SIG = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
       np.array([[1, 0], [0, -1]], complex)]


def gammas():
    g = []
    for k in range(3):
        m = np.zeros((4, 4), complex)
        m[:2, 2:] = -1j * SIG[k]
        m[2:, :2] = 1j * SIG[k]
        g.append(m)
    m = np.zeros((4, 4), complex)
    m[:2, 2:] = np.eye(2)
    m[2:, :2] = np.eye(2)
    g.append(m)
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def coords(dims):
    nx, ny, nz, nt = dims
    out = []
    for t in range(nt):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    out.append((x, y, z, t))
    return out


def lex(dims, c):
    nx, ny, nz, nt = dims
    return c[0] + nx * (c[1] + ny * (c[2] + nz * c[3]))


def dense_dw(dims, U, m0):
    """Dense D_w of Eq. 2.  U: float64 host-layout gauge array."""
    g, _ = gammas()
    V = int(np.prod(dims))
    Uc = U.view(np.complex128).reshape(V, 4, 3, 3)
    D = np.zeros((V * 12, V * 12), complex)
    eye4 = np.eye(4)
    for site, c in enumerate(coords(dims)):
        D[site * 12:(site + 1) * 12, site * 12:(site + 1) * 12] += (4.0 - m0) * np.eye(12)
        for mu in range(4):
            cf = list(c)
            cf[mu] = (cf[mu] + 1) % dims[mu]
            cb = list(c)
            cb[mu] = (cb[mu] - 1) % dims[mu]
            xf, xb = lex(dims, cf), lex(dims, cb)
            D[site * 12:(site + 1) * 12, xf * 12:(xf + 1) * 12] += -0.5 * np.kron(eye4 - g[mu], Uc[site, mu])
            D[site * 12:(site + 1) * 12, xb * 12:(xb + 1) * 12] += -0.5 * np.kron(
                eye4 + g[mu], Uc[xb, mu].conj().T)
    return D


def lmats(ns, m0, mq):
    """L+ and L- of Eq. 4 (0-based s)."""
    lp = np.zeros((ns, ns))
    for s in range(ns):
        if s > 0:
            lp[s, s - 1] = 1.0
        else:
            lp[0, ns - 1] = -mq / (2.0 * m0)
    return lp, lp.T.copy()


def dense_L(ns, m0, mq):
    """L = P+ L+ + P- L- as a (4 Ns) x (4 Ns) matrix indexed (s, spin)."""
    _, g5 = gammas()
    pp, pm = 0.5 * (np.eye(4) + g5), 0.5 * (np.eye(4) - g5)
    lp, lm = lmats(ns, m0, mq)
    return np.kron(lp, pp) + np.kron(lm, pm)


def dense_d5(dims, ns, U, m0, mq, omega, sigma):
    """Dense D = D_w (omega + sigma L) + (1 - L) (Eq. 5), index (site, s, spin, colour)."""
    V = int(np.prod(dims))
    dw = dense_dw(dims, U, m0).reshape(V, 4, 3, V, 4, 3)       # [x, alpha, a, y, gamma, b]
    L = dense_L(ns, m0, mq).reshape(ns, 4, ns, 4)              # [s, alpha, t, beta]
    eye_s4 = np.einsum("st,pq->sptq", np.eye(ns), np.eye(4))
    # omega + sigma L: omega_s on the diagonal, row s of L scaled by sigma_s
    W = np.asarray(omega)[:, None, None, None] * eye_s4 + np.asarray(sigma)[:, None, None, None] * L
    # (D_w x 1_s)(W x 1_site x 1_colour): sum over the intermediate spin gamma
    dwW = np.einsum("xpaygb,sgtq->xspaytqb", dw, W)
    block = np.einsum("xy,sptq,ab->xspaytqb", np.eye(V), eye_s4 - L, np.eye(3))
    n = V * ns * 12
    return dwW.reshape(n, n) + block.reshape(n, n)
