"""Failure detection without a GPU fault: the hop kernels' bounded waits for their TMA copies.

With dwf_debug_set_wait(skip_copies=True) the hop kernels of a context issue no copies, so
nothing completes the mbarrier they wait on and every wait runs out after its bound (a few
thousand polls here).  The kernel then sets the context's error word and returns; the call
must report DWF_ETIMEOUT, and once the hook is cleared the same context must give the
oracle's results again.  Nothing faults, traps or hangs: every wait ends by its bound."""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def case(gpu_lib):
    dims, ns, mq = (4, 4, 2, 4), 8, 0.05
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=91)
    ctx = gpu_lib.Context(dims, ns, M0, mq, om, sg, U)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    x = inputs.gaussian_source(dims, ns, seed=92)
    yield dict(dims=dims, ns=ns, mq=mq, om=om, sg=sg, U=U, ctx=ctx, mp=mp, mm=mm, x=x)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_operator_reports_timeout_and_context_recovers(gpu_lib, case, prec):
    dwf = gpu_lib
    h = case["ctx"].h
    want = oracle.ccdag_op(case["dims"], case["ns"], case["U"], case["mp"], case["mm"], 1, case["x"])
    dwf.dwf_debug_set_wait(h, 4096, skip_copies=True)
    try:
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_apply_eo(h, dwf.OP_CCDAG, prec, 1, case["x"])
        assert e.value.status == dwf.DWF_ETIMEOUT
    finally:
        dwf.dwf_debug_set_wait(h, 0, skip_copies=False)
    got = dwf.dwf_apply_eo(h, dwf.OP_CCDAG, prec, 1, case["x"])
    assert rel(got, want) < {0: 1e-12, 1: 1e-5, 3: 3e-2}[prec]


def test_solve_reports_timeout_and_context_recovers(gpu_lib, case):
    dwf = gpu_lib
    h = case["ctx"].h
    eta = inputs.gaussian_source(case["dims"], case["ns"], seed=93)
    dwf.dwf_debug_set_wait(h, 4096, skip_copies=True)
    try:
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_solve(h, eta)
        assert e.value.status == dwf.DWF_ETIMEOUT
    finally:
        dwf.dwf_debug_set_wait(h, 0, skip_copies=False)
    psi, st = dwf.dwf_solve(h, eta)
    res = np.linalg.norm(eta - oracle.dfull(case["dims"], case["ns"], case["U"], M0, case["mq"], case["om"],
                                            case["sg"], psi)) / np.linalg.norm(eta)
    assert st["converged"] == 1 and res <= 1e-10


def test_default_bound_is_restored(gpu_lib, case):
    """A bound of 0 restores the default; results with the default bound are unchanged."""
    dwf = gpu_lib
    h = case["ctx"].h
    a = dwf.dwf_apply_eo(h, dwf.OP_C, dwf.PREC_F32, 1, case["x"])
    dwf.dwf_debug_set_wait(h, 1 << 16, skip_copies=False)
    b = dwf.dwf_apply_eo(h, dwf.OP_C, dwf.PREC_F32, 1, case["x"])
    dwf.dwf_debug_set_wait(h, 0, skip_copies=False)
    assert np.array_equal(a, b)
