"""Optimal domain-wall weights (sigma = omega): the oracle pinned to the mathematics that
defines it, and the library's own construction (dwf_optimal_weights, host code behind the
C-ABI) checked against the oracle.

The weights make S = (1 - T)/(1 + T), T = prod_s (1 - omega_s lam)/(1 + omega_s lam), the
best uniform approximation of sgn on [lmin, lmax].  Pins: the closed form for Ns = 1
(S = omega lam, so omega = 2/(lmin + lmax) and delta = (lmax - lmin)/(lmax + lmin)); the
alternation theorem (the error 1 - S reaches +-delta with alternating signs at exactly
Ns + 1 points); local optimality (no perturbation of the weights lowers max |1 - S|); and
delta falling as Ns grows; and Zolotarev's closed-form solution in elliptic functions.
"""
import numpy as np
import pytest

from oracle import weights as W


@pytest.fixture(scope="module")
def lib():
    from paper_1101_0423_gb300 import build, dwf
    build.build()
    return dwf.load()

CASES = [(2, 0.05, 6.0), (3, 0.1, 5.0), (5, 0.05, 6.0), (8, 0.02, 7.0), (12, 0.05, 6.0), (16, 0.05, 6.0)]


def dense_error(omega, lmin, lmax, n=400001):
    g = np.exp(np.linspace(np.log(lmin), np.log(lmax), n))
    return g, W.error(omega, g)


def test_one_slice_closed_form():
    for lmin, lmax in [(0.05, 6.0), (0.3, 2.0), (1e-3, 10.0)]:
        om, d = W.optimal_weights(1, lmin, lmax)
        assert om[0] == pytest.approx(2.0 / (lmin + lmax), rel=1e-12)
        assert d == pytest.approx((lmax - lmin) / (lmax + lmin), rel=1e-12)


@pytest.mark.parametrize("ns,lmin,lmax", CASES)
def test_error_alternates_at_ns_plus_one_points(ns, lmin, lmax):
    om, d = W.optimal_weights(ns, lmin, lmax)
    g, e = dense_error(om, lmin, lmax)
    assert np.max(np.abs(e)) == pytest.approx(d, rel=1e-8)
    # one extremum of |e| on each interval between sign changes, all of size delta
    sign = np.sign(e)
    cuts = np.flatnonzero(sign[1:] != sign[:-1])
    assert len(cuts) == ns  # T has Ns zeros in the interval
    bounds = np.concatenate([[0], cuts + 1, [len(g)]])
    peaks = np.array([e[a:b][np.argmax(np.abs(e[a:b]))] for a, b in zip(bounds[:-1], bounds[1:])])
    assert np.allclose(np.abs(peaks), d, rtol=1e-6)
    assert np.all(np.sign(peaks) == (-1.0) ** np.arange(ns + 1))


@pytest.mark.parametrize("ns,lmin,lmax", CASES[:4])
def test_no_perturbation_lowers_the_deviation(ns, lmin, lmax):
    om, d = W.optimal_weights(ns, lmin, lmax)
    rng = np.random.default_rng(ns)
    for _ in range(20):
        trial = om * np.exp(1e-3 * rng.standard_normal(ns))
        _, e = dense_error(trial, lmin, lmax, 100001)
        assert np.max(np.abs(e)) > d * (1 - 1e-9)


def zolotarev(ns, lmin, lmax):
    """Zolotarev's solution, in elliptic functions, written independently of the oracle's
    Remez exchange.  Among T(lam) = prod_j (p_j - lam)/(p_j + lam), the one of least
    max |T| on [lmin, lmax] has the zeros p_j = lmax dn((2j - 1) K / (2 Ns), k), with modulus
    k^2 = 1 - (lmin/lmax)^2 and K = K(k) (Zolotarev's third problem, the same minimax as
    the optimal shifts of the ADI iteration); |T| then equioscillates with T(lmin) = delta_T.
    S_T = (1 - T)/(1 + T) spans [m, 1/m], m = (1 - delta_T)/(1 + delta_T), so the multiple
    C S_T with C = 2 m / (1 + m^2) spans [1 - delta, 1 + delta], delta = 2 delta_T/(1 + delta_T^2),
    touching both ends at the Ns + 1 alternation points: the best uniform approximation of
    sgn in the (1 - T)/(1 + T) family (a constant multiple of an odd rational of this type is
    again of this type).  Returns (S as a function of lam, delta)."""
    from scipy import special
    m_par = 1.0 - (lmin / lmax) ** 2                     # scipy takes the parameter k^2
    u = (2 * np.arange(1, ns + 1) - 1) * special.ellipk(m_par) / (2 * ns)
    p = lmax * special.ellipj(u, m_par)[2]               # dn
    def T(lam):
        lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
        return np.prod((p - lam[:, None]) / (p + lam[:, None]), axis=1)
    dT = abs(T(lmin)[0])
    m = (1.0 - dT) / (1.0 + dT)
    C = 2.0 * m / (1.0 + m * m)
    return (lambda lam: C * (1.0 - T(lam)) / (1.0 + T(lam))), 2.0 * dT / (1.0 + dT * dT)


@pytest.mark.parametrize("ns,lmin,lmax", [(1, 0.05, 6.0), (4, 0.05, 6.2), (8, 0.05, 6.2), (8, 0.02, 7.0),
                                          (16, 0.05, 6.2), (16, 0.3, 2.0), (5, 0.1, 5.0)])
def test_oracle_matches_zolotarev_closed_form(ns, lmin, lmax):
    """The oracle's weights give the same S(lam) and delta as Zolotarev's closed form (the
    best approximation is unique, so equal S on the interval fixes the weights)."""
    S_z, d_z = zolotarev(ns, lmin, lmax)
    om, d = W.optimal_weights(ns, lmin, lmax)
    g = np.exp(np.linspace(np.log(lmin), np.log(lmax), 100001))
    assert d == pytest.approx(d_z, rel=1e-9)
    assert np.max(np.abs((1.0 - W.error(om, g)) - S_z(g))) < 1e-10


def test_zolotarev_closed_form_alternates():
    """Check on the closed form itself: its error reaches +-delta with alternating signs at
    Ns + 1 points (a mistyped modulus or argument of dn would break this)."""
    ns, lmin, lmax = 8, 0.05, 6.2
    S_z, d_z = zolotarev(ns, lmin, lmax)
    g = np.exp(np.linspace(np.log(lmin), np.log(lmax), 400001))
    e = 1.0 - S_z(g)
    assert np.max(np.abs(e)) == pytest.approx(d_z, rel=1e-9)
    sign = np.sign(e)
    cuts = np.flatnonzero(sign[1:] != sign[:-1])
    assert len(cuts) == ns
    bounds = np.concatenate([[0], cuts + 1, [len(g)]])
    peaks = np.array([e[a:b][np.argmax(np.abs(e[a:b]))] for a, b in zip(bounds[:-1], bounds[1:])])
    assert np.allclose(np.abs(peaks), d_z, rtol=1e-6)


def test_deviation_falls_with_ns():
    ds = [W.optimal_weights(ns, 0.05, 6.0)[1] for ns in (1, 2, 4, 8, 16)]
    assert all(b < a for a, b in zip(ds, ds[1:]))
    assert ds[-1] < 1e-4


def test_weights_lie_in_the_inverse_spectrum():
    om, _ = W.optimal_weights(10, 0.05, 6.0)
    assert np.all(np.diff(om) < 0)
    assert np.all(om > 1.0 / 6.0) and np.all(om < 1.0 / 0.05)


@pytest.mark.parametrize("ns,lmin,lmax", [(1, 0.05, 6.0)] + CASES + [(32, 0.02, 7.0)])
def test_library_matches_the_oracle(lib, ns, lmin, lmax):
    from paper_1101_0423_gb300 import dwf
    om_lib, d_lib = dwf.dwf_optimal_weights(ns, lmin, lmax)
    om_or, d_or = W.optimal_weights(ns, lmin, lmax)
    assert np.max(np.abs(om_lib - om_or) / om_or) < 1e-8
    assert d_lib == pytest.approx(d_or, rel=1e-7)


@pytest.mark.parametrize("args", [(0, 0.05, 6.0), (65, 0.05, 6.0), (4, 0.0, 6.0), (4, 6.0, 0.05), (4, -1.0, 2.0)])
def test_library_rejects_invalid_ranges(lib, args):
    from paper_1101_0423_gb300 import dwf
    with pytest.raises(dwf.DwfError) as e:
        dwf.dwf_optimal_weights(*args)
    assert e.value.status == dwf.DWF_EINVAL
