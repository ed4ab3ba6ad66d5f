"""Optimal domain-wall weights (test infrastructure: only tests and the benchmark's CPU
legs import this module).

With sigma = omega (the optimal domain-wall operator of Eq. 1) the five-dimensional
operator reduces, in four dimensions, to one built on the sign-function approximation

    S(lam) = (1 - T(lam)) / (1 + T(lam)),   T(lam) = prod_s (1 - omega_s lam) / (1 + omega_s lam),

with lam over the spectrum [lmin, lmax] of |H_w|.  Sec. 2.1 names the goal of these weights
(chiral symmetry as good as Ns slices allow) and takes them from a cited formula that it
does not print.  Reading: the
optimal weights make S the best uniform approximation of sgn on [lmin, lmax], i.e. they
minimize delta = max |1 - S(lam)|.  By the alternation theorem the error e = 1 - S of the
optimum takes the value +-delta, with alternating signs, at Ns + 1 points.

This oracle finds them by the Remez exchange, written out plainly: at Ns + 1 reference
points solve e(lam_i) = (-1)^i delta for the Ns zeros x_s = 1 / omega_s of T and delta
(scipy's root finder, in the zeros' logarithms); move each reference point to the extremum of |e|
between consecutive zeros, located on a dense logarithmic grid and refined by a bounded
1-D maximisation; repeat until the extrema agree.  Parity pins (tests/test_optimal_weights.py):
Zolotarev's closed-form solution in Jacobi elliptic functions (S(lam) and delta agree), the
closed form for Ns = 1, the alternation of the result, local optimality against
perturbations, and delta decreasing with Ns.
"""
from __future__ import annotations

import numpy as np
from scipy import optimize


def error(omega, lam):
    """e(lam) = 1 - S(lam) = 2 T / (1 + T) for the weights omega."""
    omega = np.asarray(omega, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    T = np.prod((1.0 - np.multiply.outer(lam, omega)) / (1.0 + np.multiply.outer(lam, omega)), axis=-1)
    return 2.0 * T / (1.0 + T)


def _extrema(x, lmin, lmax, grid):
    """Abscissae of the extreme |e| on each of the Ns + 1 intervals cut by the zeros x."""
    edges = np.concatenate([[lmin], np.sort(x), [lmax]])
    omega = 1.0 / x
    pts = []
    for a, b in zip(edges[:-1], edges[1:]):
        g = np.exp(np.linspace(np.log(a), np.log(b), grid))
        k = int(np.argmax(np.abs(error(omega, g))))
        lo, hi = g[max(k - 1, 0)], g[min(k + 1, grid - 1)]
        if k == 0 or k == grid - 1:  # the extremum is an end of the whole interval
            pts.append(g[k])
            continue
        r = optimize.minimize_scalar(lambda t: -abs(error(omega, np.exp(t))), bounds=(np.log(lo), np.log(hi)),
                                     method="bounded", options={"xatol": 1e-14})
        pts.append(float(np.exp(r.x)))
    return np.array(pts)


def optimal_weights(ns, lmin, lmax, tol=1e-12, max_rounds=60, grid=4001):
    """The weights omega_s (decreasing along s) and delta = max |1 - S| on [lmin, lmax]."""
    if ns < 1 or not (0.0 < lmin < lmax):
        raise ValueError("need ns >= 1 and 0 < lmin < lmax")
    ratio = lmax / lmin
    x = lmin * ratio ** ((np.arange(ns) + 0.5) / ns)
    ref = lmin * ratio ** (np.arange(ns + 1) / ns)
    signs = (-1.0) ** np.arange(ns + 1)
    delta = float(np.max(np.abs(error(1.0 / x, ref))))

    def equations(v, ref):  # e(lam_i) - (-1)^i delta, in the zeros' logarithms and delta
        return error(np.exp(-v[:ns]), ref) - signs * v[ns]

    for _ in range(max_rounds):
        sol = optimize.root(equations, np.concatenate([np.log(x), [delta]]), args=(ref,), method="hybr",
                            options={"xtol": 1e-15})
        x, delta = np.sort(np.exp(sol.x[:ns])), float(sol.x[ns])
        ref = _extrema(x, lmin, lmax, grid)
        ext = np.abs(error(1.0 / x, ref))
        if ext.max() - ext.min() <= tol * ext.max():
            break
    else:
        raise RuntimeError("Remez exchange did not converge")
    omega = np.sort(1.0 / x)[::-1]
    return omega, float(np.max(np.abs(error(omega, ref))))
