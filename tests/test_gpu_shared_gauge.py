"""Gauge fields shared by handle (dwf_gauge_create / dwf_attach_gauge) through the C-ABI.

Contexts of different Ns, masses and weights attached to one device-resident gauge object
must give exactly the results of contexts that loaded their own copy (the same links, the
same kernels); the object outlives the caller's reference until its last context goes;
mismatched lattices are refused.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8
DIMS = (4, 4, 6, 4)


@pytest.fixture(scope="module")
def field(gpu_lib):
    return gpu_lib, inputs.gauge_field(DIMS, 0.5, seed=61)


@pytest.mark.parametrize("ns,kind,mq", [(8, "shamir", 0.05), (12, "cosine", 0.02), (6, "borici", 0.1)])
def test_attached_context_matches_private_copy(field, ns, kind, mq):
    dwf, U = field
    om, sg = inputs.weights(kind, ns)
    g = dwf.dwf_gauge_create(DIMS, U)
    try:
        x = inputs.gaussian_source(DIMS, ns, seed=62)
        eta = inputs.gaussian_source(DIMS, ns, seed=63)
        with dwf.Context(DIMS, ns, M0, mq, om, sg, gauge=g) as shared, \
                dwf.Context(DIMS, ns, M0, mq, om, sg, U=U) as private:
            for prec in (0, 1, 3):
                a = dwf.dwf_apply_eo(shared.h, dwf.OP_CCDAG, prec, 1, x)
                b = dwf.dwf_apply_eo(private.h, dwf.OP_CCDAG, prec, 1, x)
                assert np.array_equal(a, b)
            psi_s, st_s = dwf.dwf_solve(shared.h, eta, tol=1e-10)
            psi_p, st_p = dwf.dwf_solve(private.h, eta, tol=1e-10)
            assert np.array_equal(psi_s, psi_p) and st_s["iters"] == st_p["iters"]
        res = np.linalg.norm(eta - oracle.dfull(DIMS, ns, U, M0, mq, om, sg, psi_s)) / np.linalg.norm(eta)
        assert res <= 1e-10
    finally:
        dwf.dwf_gauge_release(g)


def test_gauge_outlives_the_callers_reference(field):
    dwf, U = field
    ns = 8
    om, sg = inputs.weights("shamir", ns)
    g = dwf.dwf_gauge_create(DIMS, U)
    a = dwf.Context(DIMS, ns, M0, 0.05, om, sg, gauge=g)
    b = dwf.Context(DIMS, ns, M0, 0.1, om, sg, gauge=g)
    dwf.dwf_gauge_release(g)          # the two contexts still hold it
    x = inputs.gaussian_source(DIMS, ns, seed=64)
    want = oracle.hop(DIMS, ns, U, 0, x)
    a.close()
    got = dwf.dwf_apply_eo(b.h, dwf.OP_DEO, dwf.PREC_F64, 0, x)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12
    b.close()


def test_load_gauge_detaches(field):
    dwf, U = field
    ns = 4
    om, sg = inputs.weights("shamir", ns)
    U2 = inputs.gauge_field(DIMS, 0.5, seed=65)
    g = dwf.dwf_gauge_create(DIMS, U)
    try:
        with dwf.Context(DIMS, ns, M0, 0.05, om, sg, gauge=g) as c:
            dwf.dwf_load_gauge(c.h, U2)   # now a private copy of another field
            x = inputs.gaussian_source(DIMS, ns, seed=66)
            got = dwf.dwf_apply_eo(c.h, dwf.OP_DEO, dwf.PREC_F64, 0, x)
            want = oracle.hop(DIMS, ns, U2, 0, x)
            assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12
    finally:
        dwf.dwf_gauge_release(g)


def test_attach_refuses_another_lattice(field):
    dwf, U = field
    om, sg = inputs.weights("shamir", 4)
    g = dwf.dwf_gauge_create(DIMS, U)
    try:
        with dwf.Context((4, 4, 4, 4), 4, M0, 0.05, om, sg) as c:
            with pytest.raises(dwf.DwfError) as e:
                dwf.dwf_attach_gauge(c.h, g)
            assert e.value.status == dwf.DWF_EINVAL
    finally:
        dwf.dwf_gauge_release(g)
