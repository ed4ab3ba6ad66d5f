"""Plain FP64 CPU oracle for the domain-wall operator and CG solver (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA path: the arithmetic lives in
``dwf_oracle.c`` (plain C, FP64, written from Sec. 2 of Chiu, Hsieh, Mao, Ogawa,
Lattice 2010), built with gcc into ``libdwf_oracle.so`` beside it.

Arrays use the host layouts described in ``dwf_oracle.h``: 5D spinors are float64
arrays of length 24*Ns*V4, gauge fields float64 arrays of length 72*V4.

Parity pins: every function here is pinned by tests/test_oracle_pins.py (Clifford
algebra, free-field momentum form, gamma5- and gamma5*R5-hermiticity, gauge
covariance, the Shamir closed form of M5, Eq. 7 vs Eq. 8, dense assembly + LU, the
Schur solve against the unpreconditioned LU solve).  The iteration and restart
counts of a mixed-precision solve are parity unpinned: the paper prints none.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwf_oracle.c")
_LIB = os.path.join(_HERE, "libdwf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: the same source on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dwf_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = bind(ctypes.CDLL(_LIB))
    return _lib


def bind(lib):
    """Declare the argument types of every oracle entry point on a loaded library."""
    P = ctypes.POINTER(ctypes.c_double)
    I4 = ctypes.POINTER(ctypes.c_int)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "or_gamma": [i, P],
        "or_dw": [I4, i, P, d, P, P],
        "or_hop": [I4, i, P, i, P, P],
        "or_hop_dag": [I4, i, P, i, P, P],
        "or_lmat": [i, d, d, P, P],
        "or_m5": [i, d, d, P, P, P, P],
        "or_s1s2": [i, d, d, P, P, P, P, P, P],
        "or_apply_s": [I4, i, P, P, i, i, P, P],
        "or_dfull": [I4, i, P, d, d, P, P, P, P],
        "or_c": [I4, i, P, P, P, i, P, P],
        "or_cdag": [I4, i, P, P, P, i, P, P],
        "or_ccdag": [I4, i, P, P, P, i, P, P],
        "or_cg": [I4, i, P, P, P, i, P, P, d, i, ctypes.POINTER(ctypes.c_int), P],
        "or_solve_full": [I4, i, P, d, d, P, P, i, P, P, d, i,
                          ctypes.POINTER(ctypes.c_int), P],
        "or_dot": [ctypes.c_long, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, name: str):
    if rc != 0:
        raise ValueError(f"oracle {name} rejected its arguments (rc={rc})")


def gamma(mu: int) -> np.ndarray:
    out = np.zeros(32)
    _check(_load().or_gamma(mu, _p(out)), "or_gamma")
    return out.view(np.complex128).reshape(4, 4)


def dw(dims, ns, U, m0, x):
    x, U = _f64(x), _f64(U)
    out = np.empty_like(x)
    _check(_load().or_dw(_dims(dims), ns, _p(U), m0, _p(x), _p(out)), "or_dw")
    return out


def hop(dims, ns, U, p, x):
    x, U = _f64(x), _f64(U)
    out = np.empty_like(x)
    _check(_load().or_hop(_dims(dims), ns, _p(U), p, _p(x), _p(out)), "or_hop")
    return out


def hop_dag(dims, ns, U, p, x):
    x, U = _f64(x), _f64(U)
    out = np.empty_like(x)
    _check(_load().or_hop_dag(_dims(dims), ns, _p(U), p, _p(x), _p(out)), "or_hop_dag")
    return out


def lmat(ns, m0, mq):
    lp, lm = np.zeros(ns * ns), np.zeros(ns * ns)
    _check(_load().or_lmat(ns, m0, mq, _p(lp), _p(lm)), "or_lmat")
    return lp.reshape(ns, ns), lm.reshape(ns, ns)


def m5(ns, m0, mq, omega, sigma):
    omega, sigma = _f64(omega), _f64(sigma)
    mp, mm = np.zeros(ns * ns), np.zeros(ns * ns)
    _check(_load().or_m5(ns, m0, mq, _p(omega), _p(sigma), _p(mp), _p(mm)), "or_m5")
    return mp.reshape(ns, ns), mm.reshape(ns, ns)


def s1s2(ns, m0, mq, omega, sigma):
    omega, sigma = _f64(omega), _f64(sigma)
    bufs = [np.zeros(ns * ns) for _ in range(4)]
    _check(_load().or_s1s2(ns, m0, mq, _p(omega), _p(sigma), *[_p(b) for b in bufs]), "or_s1s2")
    return [b.reshape(ns, ns) for b in bufs]


def apply_s(dims, ns, mp, mm, x, transpose=False, parity=-1):
    x = _f64(x)
    mp, mm = _f64(mp).reshape(-1), _f64(mm).reshape(-1)
    out = np.empty_like(x)
    _check(_load().or_apply_s(_dims(dims), ns, _p(mp), _p(mm), int(bool(transpose)), parity,
                              _p(x), _p(out)), "or_apply_s")
    return out


def dfull(dims, ns, U, m0, mq, omega, sigma, x):
    x, U, omega, sigma = _f64(x), _f64(U), _f64(omega), _f64(sigma)
    out = np.empty_like(x)
    _check(_load().or_dfull(_dims(dims), ns, _p(U), m0, mq, _p(omega), _p(sigma), _p(x),
                            _p(out)), "or_dfull")
    return out


def _cop(name, dims, ns, U, mp, mm, p, x):
    x, U = _f64(x), _f64(U)
    mp, mm = _f64(mp).reshape(-1), _f64(mm).reshape(-1)
    out = np.empty_like(x)
    _check(getattr(_load(), name)(_dims(dims), ns, _p(U), _p(mp), _p(mm), p, _p(x), _p(out)), name)
    return out


def c_op(dims, ns, U, mp, mm, p, x):
    return _cop("or_c", dims, ns, U, mp, mm, p, x)


def cdag_op(dims, ns, U, mp, mm, p, x):
    return _cop("or_cdag", dims, ns, U, mp, mm, p, x)


def ccdag_op(dims, ns, U, mp, mm, p, x):
    return _cop("or_ccdag", dims, ns, U, mp, mm, p, x)


def cg(dims, ns, U, mp, mm, p, b, tol=1e-12, maxiter=100000, x0=None):
    """CG on C C^dagger (Algorithm 1).  Returns (x, iters, true relative residual)."""
    b, U = _f64(b), _f64(U)
    mp, mm = _f64(mp).reshape(-1), _f64(mm).reshape(-1)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    _check(_load().or_cg(_dims(dims), ns, _p(U), _p(mp), _p(mm), p, _p(b), _p(x), tol, maxiter,
                         ctypes.byref(it), ctypes.byref(rr)), "or_cg")
    return x, it.value, rr.value


def solve_full(dims, ns, U, m0, mq, omega, sigma, eta, p=1, tol=1e-12, maxiter=100000):
    """Solve D psi = eta through the Schur complement (Eq. 10).  Returns (psi, iters, relres)."""
    eta, U, omega, sigma = _f64(eta), _f64(U), _f64(omega), _f64(sigma)
    psi = np.empty_like(eta)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    _check(_load().or_solve_full(_dims(dims), ns, _p(U), m0, mq, _p(omega), _p(sigma), p,
                                 _p(eta), _p(psi), tol, maxiter, ctypes.byref(it),
                                 ctypes.byref(rr)), "or_solve_full")
    return psi, it.value, rr.value


def dot(a, b) -> complex:
    a, b = _f64(a), _f64(b)
    re, im = ctypes.c_double(0), ctypes.c_double(0)
    _check(_load().or_dot(a.size, _p(a), _p(b), ctypes.byref(re), ctypes.byref(im)), "or_dot")
    return complex(re.value, im.value)
