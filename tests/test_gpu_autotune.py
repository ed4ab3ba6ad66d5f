"""The launch-shape autotuner on the GPU, through the C-ABI.

The first solve of each (precision, Ns, volume class) times the candidate launch shapes of
the inner CG's three hop kernels and keeps the fastest; dwf_tuned_shape then reports a
tuned shape for each.  Solves with tuned shapes meet the oracle-recomputed residual, and
agree with solves that keep the default shapes (no_autotune) within the conditioning bound
of that residual: only the order of the reductions' block sums differs.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8


@pytest.mark.parametrize("ns", [8, 12, 24, 32])
def test_solve_tunes_every_inner_hop_kernel(gpu_lib, ns):
    dwf = gpu_lib
    dims, mq = (4, 4, 4, 8), 0.05
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.5, seed=70 + ns)
    eta = inputs.gaussian_source(dims, ns, seed=71 + ns)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        psi_d, st_d = dwf.dwf_solve(ctx.h, eta, tol=1e-10, no_autotune=1)
        psi, st = dwf.dwf_solve(ctx.h, eta, tol=1e-10)
        for kc in (dwf.KC_HOP_M5, dwf.KC_HOP_XPAY, dwf.KC_HOP_UPDATE):
            threads, persistent, tuned = dwf.dwf_tuned_shape(ctx.h, dwf.PREC_F32, kc)
            assert tuned, f"class {kc} not tuned at Ns={ns}"
            spb = max(1, min(64, threads // ns))
            assert threads in (64, 128, 256) and spb * ns <= 256
        psi2, st2 = dwf.dwf_solve(ctx.h, eta, tol=1e-10)   # tuned shapes are kept: same result
        assert np.array_equal(psi, psi2)
    res = np.linalg.norm(eta - oracle.dfull(dims, ns, U, M0, mq, om, sg, psi)) / np.linalg.norm(eta)
    assert res <= 1e-10 and st["converged"] == 1
    assert np.linalg.norm(psi - psi_d) / np.linalg.norm(psi_d) < 1e-6


def test_untuned_query_reports_the_default(gpu_lib):
    dwf = gpu_lib
    dims, ns = (4, 4, 4, 4), 7
    om, sg = inputs.weights("shamir", ns)
    with dwf.Context(dims, ns, M0, 0.05, om, sg, inputs.gauge_field(dims, 0.5, seed=79)) as ctx:
        threads, persistent, tuned = dwf.dwf_tuned_shape(ctx.h, dwf.PREC_BF16, dwf.KC_HOP_XPAY)
        assert not tuned and threads == 128 and persistent
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_tuned_shape(ctx.h, dwf.PREC_F64, dwf.KC_HOP_M5)
        assert e.value.status == dwf.DWF_EINVAL
