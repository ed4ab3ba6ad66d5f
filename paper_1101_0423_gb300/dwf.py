"""Thin ctypes binding of the C-ABI in include/dwf.h (argument marshalling only).

Every function keeps the C name.  Host arrays are float64 numpy arrays in the host
layouts of include/dwf.h; the ``*_dev`` functions take device pointers (ints, or any
object with ``data_ptr()`` such as a torch CUDA tensor) and an optional CUDA stream
(an int handle or an object with ``cuda_stream``).  Errors raise :class:`DwfError`
carrying the status and the library's message.  There is no CPU fallback: if the
CUDA library cannot be built or loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdwf_gb300.so")

OP_DEO, OP_DOE, OP_M5, OP_M5T, OP_C, OP_CDAG, OP_CCDAG, OP_DFULL, OP_DW = range(9)
PREC_F64, PREC_F32, PREC_F16, PREC_BF16 = range(4)
MODE_AUTO, MODE_RELIABLE, MODE_DEFECT = range(3)
SYS_FULL, SYS_NORMAL = range(2)
KC_NAMES = ["hop_m5", "hop_xpay", "hop_update", "smix_p", "f64", "other"]
KC_HOP_M5, KC_HOP_XPAY, KC_HOP_UPDATE = range(3)
STATUS = ["DWF_OK", "DWF_EINVAL", "DWF_ENOMEM", "DWF_ENOCONV", "DWF_EBUSY", "DWF_EAGAIN",
          "DWF_ETIMEOUT", "DWF_ECUDA", "DWF_ENOGAUGE", "DWF_ECOMM"]
DWF_OK, DWF_EINVAL, DWF_ENOMEM, DWF_ENOCONV, DWF_EBUSY, DWF_EAGAIN, DWF_ETIMEOUT, DWF_ECUDA, \
    DWF_ENOGAUGE, DWF_ECOMM = range(10)


class DwfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("delta", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("mode", ctypes.c_int), ("system", ctypes.c_int),
                ("schur_parity", ctypes.c_int), ("check_every", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("profile", ctypes.c_int), ("stall_iters", ctypes.c_int),
                ("schur_target_pct", ctypes.c_int), ("use_x0", ctypes.c_int), ("no_autotune", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("mode_used", ctypes.c_int),
                ("converged", ctypes.c_int), ("true_res", ctypes.c_double),
                ("true_res_full", ctypes.c_double), ("flops", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("class_ms", ctypes.c_double * 6),
                ("class_launches", ctypes.c_int * 6), ("kernel_launches", ctypes.c_longlong),
                ("bytes_hop_m5", ctypes.c_double), ("inner_prec_used", ctypes.c_int),
                ("escalations", ctypes.c_int), ("reserved", ctypes.c_double * 2)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("class_ms", "class_launches", "reserved")}
        d["class_ms"] = {n: self.class_ms[i] for i, n in enumerate(KC_NAMES)}
        d["class_launches"] = {n: self.class_launches[i] for i, n in enumerate(KC_NAMES)}
        return d


class Partition(ctypes.Structure):
    _fields_ = [("global_dims", ctypes.c_int * 4), ("grid", ctypes.c_int * 4), ("coord", ctypes.c_int * 4)]


# callbacks of dwf_part_comm (the transport between parts held by different processes)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                               ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t))
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


class PartComm(ctypes.Structure):
    _fields_ = [("user", ctypes.c_void_p), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN)]


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_gb", ctypes.c_double), ("max_inflight", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class Request(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("Ns", ctypes.c_int), ("m0", ctypes.c_double),
                ("mq", ctypes.c_double), ("omega", ctypes.POINTER(ctypes.c_double)),
                ("sigma", ctypes.POINTER(ctypes.c_double)), ("gauge", ctypes.c_int),
                ("rhs", ctypes.POINTER(ctypes.c_double)), ("params", SolveParams)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stats", SolveStats), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("in_flight", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("hbm_reserved_gb", ctypes.c_double),
                ("cancelled", ctypes.c_longlong), ("batched", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(build_if_missing: bool = True):
    """Load libdwf_gb300.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library missing: {LIB_PATH}")
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "dwf_create": ([ip, i, d, d, dp, dp, ctypes.POINTER(vp)], i),
        "dwf_destroy": ([vp], i),
        "dwf_load_gauge": ([vp, dp], i),
        "dwf_load_gauge_dev": ([vp, vp, vp], i),
        "dwf_gauge_create": ([ip, dp, ctypes.POINTER(vp)], i),
        "dwf_gauge_create_dev": ([ip, vp, vp, ctypes.POINTER(vp)], i),
        "dwf_gauge_release": ([vp], i),
        "dwf_attach_gauge": ([vp, vp], i),
        "dwf_apply_eo": ([vp, i, i, i, dp, dp], i),
        "dwf_apply_eo_dev": ([vp, i, i, i, vp, vp, vp], i),
        "dwf_apply_eo_dev_static": ([vp, i, i, i, vp, vp, vp], i),
        "dwf_solve": ([vp, dp, dp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats)], i),
        "dwf_solve_dev": ([vp, vp, vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp], i),
        "dwf_propagator": ([vp, ip, ctypes.POINTER(SolveParams), dp, ctypes.POINTER(SolveStats)], i),
        "dwf_propagator_dev": ([vp, ip, ctypes.POINTER(SolveParams), vp, ctypes.POINTER(SolveStats), vp], i),
        "dwf_solve_batch": ([vp, i, dp, dp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats)], i),
        "dwf_solve_batch_dev": ([vp, i, vp, vp, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp],
                                i),
        "dwf_last_error": ([vp], ctypes.c_char_p),
        "dwf_status_string": ([i], ctypes.c_char_p),
        "dwf_solve_params_default": ([ctypes.POINTER(SolveParams)], None),
        "dwf_server_params_default": ([ctypes.POINTER(ServerParams)], None),
        "dwf_server_create": ([ctypes.POINTER(ServerParams), ctypes.POINTER(vp)], i),
        "dwf_server_destroy": ([vp], i),
        "dwf_server_add_gauge": ([vp, ip, dp, ip], i),
        "dwf_submit": ([vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], i),
        "dwf_poll": ([vp, ctypes.c_uint64, dp, ctypes.POINTER(Result)], i),
        "dwf_server_get_stats": ([vp, ctypes.POINTER(ServerStats)], i),
        "dwf_optimal_weights": ([i, d, d, dp, dp], i),
        "dwf_debug_set_wait": ([vp, ctypes.c_uint, i], i),
        "dwf_tuned_shape": ([vp, i, i, ip, ip], i),
        "dwf_create_part": ([ctypes.POINTER(Partition), i, d, d, dp, dp, ctypes.POINTER(vp)], i),
        "dwf_load_gauge_part": ([vp, dp], i),
        "dwf_part_apply": ([i, ctypes.POINTER(vp), i, i, i, dp, dp], i),
        "dwf_part_solve": ([i, ctypes.POINTER(vp), dp, dp, ctypes.POINTER(SolveParams),
                            ctypes.POINTER(SolveStats)], i),
        "dwf_solve_ragged": ([i, ctypes.POINTER(vp), ctypes.POINTER(dp), ctypes.POINTER(dp),
                              ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats)], i),
        "dwf_solve_ragged_dev": ([i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                  ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), vp], i),
        "dwf_part_apply_comm": ([vp, ctypes.POINTER(PartComm), i, i, i, dp, dp], i),
        "dwf_part_solve_comm": ([vp, ctypes.POINTER(PartComm), dp, dp, ctypes.POINTER(SolveParams),
                                 ctypes.POINTER(SolveStats)], i),
        "dwf_cancel": ([vp, ctypes.c_uint64], i),
        "dwf_server_set_admission": ([vp, i], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("expected a device pointer (int) or an object with data_ptr()")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(ctx, st):
    if st != DWF_OK:
        msg = load().dwf_last_error(ctx).decode() if ctx else ""
        raise DwfError(st, msg)


def dwf_solve_params_default() -> SolveParams:
    p = SolveParams()
    load().dwf_solve_params_default(ctypes.byref(p))
    return p


def dwf_optimal_weights(Ns, lambda_min, lambda_max):
    """(omega, delta): the optimal domain-wall weights for |H_w| in [lambda_min, lambda_max]
    (decreasing) and the deviation max |1 - S| of their sign-function approximation."""
    omega = np.zeros(max(int(Ns), 1))
    delta = ctypes.c_double(0.0)
    st = load().dwf_optimal_weights(int(Ns), float(lambda_min), float(lambda_max), _dp(omega), ctypes.byref(delta))
    if st != DWF_OK:
        raise DwfError(st, "dwf_optimal_weights: invalid range or no convergence")
    return omega[:int(Ns)], delta.value


def dwf_create(dims, Ns, m0, mq, omega, sigma):
    """Returns an opaque context handle (int)."""
    lib = load()
    omega, sigma = _f64(omega), _f64(sigma)
    out = ctypes.c_void_p()
    st = lib.dwf_create((ctypes.c_int * 4)(*[int(v) for v in dims]), int(Ns), float(m0), float(mq),
                        _dp(omega), _dp(sigma), ctypes.byref(out))
    if st != DWF_OK:
        raise DwfError(st, "dwf_create rejected its arguments or could not allocate")
    return out.value


def dwf_destroy(ctx):
    _check(None, load().dwf_destroy(ctx))


def dwf_load_gauge(ctx, U):
    U = _f64(U)
    _check(ctx, load().dwf_load_gauge(ctx, _dp(U)))


def dwf_load_gauge_dev(ctx, d_U, stream=None):
    _check(ctx, load().dwf_load_gauge_dev(ctx, _ptr(d_U), _stream(stream)))


def dwf_gauge_create(dims, U):
    """A device-resident gauge field shareable by handle among contexts of this lattice."""
    U = _f64(U)
    out = ctypes.c_void_p()
    st = load().dwf_gauge_create((ctypes.c_int * 4)(*[int(v) for v in dims]), _dp(U), ctypes.byref(out))
    if st != DWF_OK:
        raise DwfError(st, "dwf_gauge_create rejected the lattice or could not allocate")
    return out.value


def dwf_gauge_create_dev(dims, d_U, stream=None):
    out = ctypes.c_void_p()
    st = load().dwf_gauge_create_dev((ctypes.c_int * 4)(*[int(v) for v in dims]), _ptr(d_U), _stream(stream),
                                     ctypes.byref(out))
    if st != DWF_OK:
        raise DwfError(st, "dwf_gauge_create_dev rejected the lattice or could not allocate")
    return out.value


def dwf_gauge_release(gauge):
    _check(None, load().dwf_gauge_release(gauge))


def dwf_attach_gauge(ctx, gauge):
    _check(ctx, load().dwf_attach_gauge(ctx, gauge))


def dwf_apply_eo(ctx, op, prec, parity, x) -> np.ndarray:
    x = _f64(x)
    out = np.empty_like(x)
    _check(ctx, load().dwf_apply_eo(ctx, int(op), int(prec), int(parity), _dp(x), _dp(out)))
    return out


def dwf_apply_eo_dev(ctx, op, prec, parity, d_in, d_out, stream=None):
    _check(ctx, load().dwf_apply_eo_dev(ctx, int(op), int(prec), int(parity), _ptr(d_in), _ptr(d_out),
                                        _stream(stream)))


def dwf_apply_eo_dev_static(ctx, op, prec, parity, d_in, d_out, stream=None):
    """Allocation-free dwf_apply_eo_dev: work fields live in the library's static device array."""
    _check(ctx, load().dwf_apply_eo_dev_static(ctx, int(op), int(prec), int(parity), _ptr(d_in), _ptr(d_out),
                                               _stream(stream)))


def _params(params=None, **kw) -> SolveParams:
    p = dwf_solve_params_default() if params is None else params
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def dwf_solve(ctx, rhs, params=None, allow_noconv=False, x0=None, **kw):
    """Returns (solution array, stats dict).  Keyword arguments override params fields; x0
    (an initial guess, same layout as the solution) starts the solve from it (use_x0)."""
    rhs = _f64(rhs)
    sol = np.empty_like(rhs) if x0 is None else _f64(x0).copy()
    p = _params(params, **kw)
    if x0 is not None:
        p.use_x0 = 1
    stats = SolveStats()
    st = load().dwf_solve(ctx, _dp(rhs), _dp(sol), ctypes.byref(p), ctypes.byref(stats))
    if not (allow_noconv and st == DWF_ENOCONV):
        _check(ctx, st)
    return sol, stats.as_dict()


def dwf_solve_dev(ctx, d_rhs, d_sol, params=None, stream=None, allow_noconv=False, **kw) -> dict:
    p = _params(params, **kw)
    stats = SolveStats()
    st = load().dwf_solve_dev(ctx, _ptr(d_rhs), _ptr(d_sol), ctypes.byref(p), ctypes.byref(stats),
                              _stream(stream))
    if not (allow_noconv and st == DWF_ENOCONV):
        _check(ctx, st)
    return stats.as_dict()


def dwf_solve_batch(ctx, rhs, params=None, allow_noconv=False, x0=None, **kw):
    """rhs: array of shape (nrhs, 24*Ns*V4) (or flat).  Returns (solutions, list of stats dicts).
    x0: initial guesses of the same shape (use_x0)."""
    rhs = _f64(rhs)
    nrhs = rhs.shape[0] if rhs.ndim > 1 else 1
    sol = np.empty_like(rhs) if x0 is None else _f64(x0).reshape(rhs.shape).copy()
    p = _params(params, **kw)
    if x0 is not None:
        p.use_x0 = 1
    stats = (SolveStats * nrhs)()
    st = load().dwf_solve_batch(ctx, nrhs, _dp(rhs), _dp(sol), ctypes.byref(p), stats)
    if not (allow_noconv and st == DWF_ENOCONV):
        _check(ctx, st)
    return sol, [stats[k].as_dict() for k in range(nrhs)]


def dwf_solve_batch_dev(ctx, nrhs, d_rhs, d_sol, params=None, stream=None, allow_noconv=False, **kw):
    p = _params(params, **kw)
    stats = (SolveStats * nrhs)()
    st = load().dwf_solve_batch_dev(ctx, int(nrhs), _ptr(d_rhs), _ptr(d_sol), ctypes.byref(p), stats,
                                    _stream(stream))
    if not (allow_noconv and st == DWF_ENOCONV):
        _check(ctx, st)
    return [stats[k].as_dict() for k in range(nrhs)]


def dwf_propagator(ctx, dims, x0, params=None, allow_noconv=False, **kw):
    """Returns (prop, stats): prop[site, alpha, a, beta, b] complex128 of shape (V4, 4, 3, 4, 3)."""
    v4 = int(np.prod(dims))
    out = np.empty(v4 * 144 * 2)
    p = _params(params, **kw)
    stats = (SolveStats * 12)()
    st = load().dwf_propagator(ctx, (ctypes.c_int * 4)(*[int(v) for v in x0]), ctypes.byref(p), _dp(out), stats)
    if not (allow_noconv and st == DWF_ENOCONV):
        _check(ctx, st)
    return out.view(np.complex128).reshape(v4, 4, 3, 4, 3), [stats[k].as_dict() for k in range(12)]


def dwf_tuned_shape(ctx, prec, kclass):
    """(threads per CTA, persistent, tuned) of an inner-CG hop kernel class for this context."""
    t, p = ctypes.c_int(0), ctypes.c_int(0)
    st = load().dwf_tuned_shape(ctx, int(prec), int(kclass), ctypes.byref(t), ctypes.byref(p))
    if st not in (DWF_OK, DWF_EAGAIN):
        _check(ctx, st)
    return t.value, bool(p.value), st == DWF_OK


def dwf_create_part(global_dims, grid, coord, Ns, m0, mq, omega, sigma):
    """A context for the block `coord` of a 4D domain decomposition (opaque handle)."""
    omega, sigma = _f64(omega), _f64(sigma)
    pt = Partition((ctypes.c_int * 4)(*global_dims), (ctypes.c_int * 4)(*grid), (ctypes.c_int * 4)(*coord))
    out = ctypes.c_void_p()
    st = load().dwf_create_part(ctypes.byref(pt), int(Ns), float(m0), float(mq), _dp(omega), _dp(sigma),
                                ctypes.byref(out))
    if st != DWF_OK:
        raise DwfError(st, "dwf_create_part rejected the decomposition or could not allocate")
    return out.value


def dwf_load_gauge_part(ctx, U_global):
    U_global = _f64(U_global)
    _check(ctx, load().dwf_load_gauge_part(ctx, _dp(U_global)))


def dwf_part_apply(parts, op, prec, parity, x) -> np.ndarray:
    """Applies op to the global host array x across all parts (faces exchanged between hops)."""
    x = _f64(x)
    out = np.empty_like(x)
    arr = (ctypes.c_void_p * len(parts))(*parts)
    _check(parts[0], load().dwf_part_apply(len(parts), arr, int(op), int(prec), int(parity), _dp(x), _dp(out)))
    return out


def dwf_part_solve(parts, rhs, params=None, allow_noconv=False, **kw):
    """Solve across the parts of a domain decomposition; (global solution, stats dict)."""
    rhs = _f64(rhs)
    sol = np.empty_like(rhs)
    p = _params(params, **kw)
    st = SolveStats()
    arr = (ctypes.c_void_p * len(parts))(*parts)
    rc = load().dwf_part_solve(len(parts), arr, _dp(rhs), _dp(sol), ctypes.byref(p), ctypes.byref(st))
    if not (allow_noconv and rc == DWF_ENOCONV):
        _check(parts[0], rc)
    return sol, st.as_dict()


def _check_set(ctxs, st):
    """Raises for a failed call on a set of contexts, with the first context's message found."""
    if st != DWF_OK:
        msg = ""
        for c in ctxs:
            msg = load().dwf_last_error(c).decode() if c else ""
            if msg:
                break
        raise DwfError(st, msg)


def dwf_solve_ragged(ctxs, rhs, params=None, allow_noconv=False, **kw):
    """One system per context (a ragged set: each context its own lattice, Ns, masses and
    weights); rhs[k] is a source of context k.  Returns (list of solutions, list of stats)."""
    n = len(ctxs)
    rhs = [_f64(r) for r in rhs]
    sol = [np.empty_like(r) for r in rhs]
    p = _params(params, **kw)
    stats = (SolveStats * n)()
    DP = ctypes.POINTER(ctypes.c_double)
    rc = load().dwf_solve_ragged(n, (ctypes.c_void_p * n)(*ctxs), (DP * n)(*[_dp(r) for r in rhs]),
                                 (DP * n)(*[_dp(x) for x in sol]), ctypes.byref(p), stats)
    if not (allow_noconv and rc == DWF_ENOCONV):
        _check_set(ctxs, rc)
    return sol, [stats[k].as_dict() for k in range(n)]


def dwf_solve_ragged_dev(ctxs, d_rhs, d_sol, params=None, stream=None, allow_noconv=False, **kw):
    """Device-array form of dwf_solve_ragged: d_rhs[k], d_sol[k] device arrays of context k."""
    n = len(ctxs)
    p = _params(params, **kw)
    stats = (SolveStats * n)()
    VP = ctypes.c_void_p
    rc = load().dwf_solve_ragged_dev(n, (VP * n)(*ctxs), (VP * n)(*[_ptr(x) for x in d_rhs]),
                                     (VP * n)(*[_ptr(x) for x in d_sol]), ctypes.byref(p), stats,
                                     _stream(stream))
    if not (allow_noconv and rc == DWF_ENOCONV):
        _check_set(ctxs, rc)
    return [stats[k].as_dict() for k in range(n)]


def part_comm(exchange, allreduce) -> PartComm:
    """A dwf_part_comm from two Python callables: exchange(send, recv) with send[k] / recv[k]
    (k = 2 mu + side) uint8 numpy views of the library's face buffers, None where nothing
    moves; allreduce(v) summing the float64 array v over all parts in place.  An exception
    in either fails the library call with DWF_ECOMM.  Keep the returned object alive while
    the library may call it."""
    def _exchange(user, send, recv, nbytes):
        try:
            s, r = [None] * 8, [None] * 8
            for k in range(8):
                n = int(nbytes[k])
                if n:
                    s[k] = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(send[k]))
                    r[k] = np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(recv[k]))
            exchange(s, r)
            return 0
        except Exception:
            return 1

    def _allreduce(user, v, n):
        try:
            allreduce(np.ctypeslib.as_array(v, shape=(int(n),)))
            return 0
        except Exception:
            return 1

    c = PartComm(None, EXCHANGE_FN(_exchange), ALLREDUCE_FN(_allreduce))
    c._keep = (_exchange, _allreduce)
    return c


def dwf_part_apply_comm(part, comm, op, prec, parity, x) -> np.ndarray:
    """dwf_part_apply for this process's part alone; x and the result are its local block."""
    x = _f64(x)
    out = np.empty_like(x)
    _check(part, load().dwf_part_apply_comm(part, ctypes.byref(comm), int(op), int(prec), int(parity), _dp(x),
                                            _dp(out)))
    return out


def dwf_part_solve_comm(part, comm, rhs, params=None, allow_noconv=False, **kw):
    """dwf_part_solve for this process's part alone; (local solution block, stats dict)."""
    rhs = _f64(rhs)
    sol = np.empty_like(rhs)
    p = _params(params, **kw)
    st = SolveStats()
    rc = load().dwf_part_solve_comm(part, ctypes.byref(comm), _dp(rhs), _dp(sol), ctypes.byref(p), ctypes.byref(st))
    if not (allow_noconv and rc == DWF_ENOCONV):
        _check(part, rc)
    return sol, st.as_dict()


def dwf_last_error(ctx) -> str:
    return load().dwf_last_error(ctx).decode()


def dwf_debug_set_wait(ctx, wait_tries=0, skip_copies=False):
    """Failure-detection hook: bound of the hop kernels' waits (mbarrier polls, 0 = default)
    and whether their TMA copies are left out so that every wait runs out."""
    _check(ctx, load().dwf_debug_set_wait(ctx, int(wait_tries), 1 if skip_copies else 0))


class Context:
    """Owns a dwf_ctx; closes it on exit."""

    def __init__(self, dims, Ns, m0, mq, omega, sigma, U=None, gauge=None):
        """U: a host gauge field copied into the context; gauge: a dwf_gauge handle to share."""
        self.dims, self.Ns = tuple(dims), int(Ns)
        self.h = dwf_create(dims, Ns, m0, mq, omega, sigma)
        if U is not None:
            dwf_load_gauge(self.h, U)
        elif gauge is not None:
            dwf_attach_gauge(self.h, gauge)

    def close(self):
        if self.h:
            dwf_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

def dwf_server_params_default() -> ServerParams:
    p = ServerParams()
    load().dwf_server_params_default(ctypes.byref(p))
    return p


def dwf_server_create(hbm_budget_gb=None, max_inflight=None):
    p = dwf_server_params_default()
    if hbm_budget_gb is not None:
        p.hbm_budget_gb = float(hbm_budget_gb)
    if max_inflight is not None:
        p.max_inflight = int(max_inflight)
    out = ctypes.c_void_p()
    st = load().dwf_server_create(ctypes.byref(p), ctypes.byref(out))
    if st != DWF_OK:
        raise DwfError(st, "dwf_server_create")
    return out.value


def dwf_server_destroy(srv):
    _check(None, load().dwf_server_destroy(srv))


def dwf_server_add_gauge(srv, dims, U) -> int:
    U = _f64(U)
    h = ctypes.c_int(-1)
    st = load().dwf_server_add_gauge(srv, (ctypes.c_int * 4)(*[int(v) for v in dims]), _dp(U), ctypes.byref(h))
    if st != DWF_OK:
        raise DwfError(st, "dwf_server_add_gauge")
    return h.value


def dwf_submit(srv, dims, Ns, m0, mq, omega, sigma, gauge, rhs, params=None, **kw) -> int:
    """Queue one solve; returns its ticket.  Keyword arguments override params fields."""
    omega, sigma, rhs = _f64(omega), _f64(sigma), _f64(rhs)
    r = Request()
    r.dims = (ctypes.c_int * 4)(*[int(v) for v in dims])
    r.Ns, r.m0, r.mq, r.gauge = int(Ns), float(m0), float(mq), int(gauge)
    r.omega, r.sigma, r.rhs = _dp(omega), _dp(sigma), _dp(rhs)
    r.params = _params(params, **kw)
    t = ctypes.c_uint64(0)
    st = load().dwf_submit(srv, ctypes.byref(r), ctypes.byref(t))
    if st != DWF_OK:
        raise DwfError(st, "dwf_submit")
    return t.value


def dwf_poll(srv, ticket, out=None):
    """None while queued or running; else (solution or None, result dict)."""
    res = Result()
    ptr = _dp(out) if out is not None else None
    st = load().dwf_poll(srv, ctypes.c_uint64(ticket), ptr, ctypes.byref(res))
    if st == DWF_EAGAIN:
        return None
    if st != DWF_OK:
        raise DwfError(st, "dwf_poll")
    return out, {"status": res.status, "stats": res.stats.as_dict(), "queue_ms": res.queue_ms,
                 "latency_ms": res.latency_ms}


def dwf_cancel(srv, ticket) -> bool:
    """Withdraw a queued request: True if it was withdrawn, False if a worker already took it."""
    st = load().dwf_cancel(srv, ctypes.c_uint64(ticket))
    if st == DWF_EBUSY:
        return False
    if st != DWF_OK:
        raise DwfError(st, "dwf_cancel")
    return True


def dwf_server_set_admission(srv, open_: bool):
    _check(None, load().dwf_server_set_admission(srv, 1 if open_ else 0))


def dwf_server_get_stats(srv) -> dict:
    s = ServerStats()
    _check(None, load().dwf_server_get_stats(srv, ctypes.byref(s)))
    return s.as_dict()
