"""4D domain decomposition through the C-ABI (dwf_create_part, dwf_load_gauge_part,
dwf_part_apply, dwf_part_solve): the lattice cut into blocks, each a part context with halo
slots, the spin-projected faces exchanged between parts before every hop, the reductions of
the solver summed over the parts.

Every operator applied across the parts must equal the oracle on the whole lattice (FP64
1e-12, FP32 1e-5, fp16 5e-3) and, in FP64 and FP32, the unpartitioned context bit for bit:
a halo slot holds the projection the receiving hop would have formed itself, so the
arithmetic is the same.  Cuts along one, two and four directions, with blocks as thin as two
sites (every site on a face), and invalid decompositions and calls are refused.  Solves
across the parts meet the oracle-recomputed true residual and agree with the whole-lattice
solve within the conditioning bound of that residual.
"""
import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8
TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}


def coords(grid):
    for t in range(grid[3]):
        for z in range(grid[2]):
            for y in range(grid[1]):
                for x in range(grid[0]):
                    yield (x, y, z, t)


def make_parts(dwf, dims, grid, ns, mq, om, sg, U, shuffle=False):
    cs = list(coords(grid))
    if shuffle:
        cs = cs[::-1]
    parts = [dwf.dwf_create_part(dims, grid, c, ns, M0, mq, om, sg) for c in cs]
    for p in parts:
        dwf.dwf_load_gauge_part(p, U)
    return parts


CASES = [((4, 4, 4, 8), (1, 1, 1, 2), 8, "cosine", 0.02),
         ((4, 4, 4, 8), (1, 1, 2, 4), 6, "shamir", 0.05),
         ((4, 4, 4, 4), (2, 2, 2, 2), 5, "borici", 0.1),
         ((8, 4, 2, 4), (2, 1, 1, 2), 16, "cosine", 0.0)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[1])) + f"_Ns{c[2]}")
def case(request, gpu_lib):
    dwf = gpu_lib
    dims, grid, ns, kind, mq = request.param
    om, sg = inputs.weights(kind, ns)
    U = inputs.gauge_field(dims, 0.5, seed=51)
    parts = make_parts(dwf, dims, grid, ns, mq, om, sg, U, shuffle=grid[0] > 1)
    whole = dwf.Context(dims, ns, M0, mq, om, sg, U)
    mp, mm = oracle.m5(ns, M0, mq, om, sg)
    x = inputs.gaussian_source(dims, ns, seed=52)
    yield dict(dwf=dwf, dims=dims, ns=ns, U=U, parts=parts, whole=whole, mp=mp, mm=mm, x=x)
    for p in parts:
        dwf.dwf_destroy(p)
    whole.close()


def _want(c, op, p):
    dwf, d, ns, U, x = c["dwf"], c["dims"], c["ns"], c["U"], c["x"]
    if op == dwf.OP_DEO:
        return oracle.hop(d, ns, U, 0, x)
    if op == dwf.OP_DOE:
        return oracle.hop(d, ns, U, 1, x)
    f = {dwf.OP_C: oracle.c_op, dwf.OP_CDAG: oracle.cdag_op, dwf.OP_CCDAG: oracle.ccdag_op}[op]
    return f(d, ns, U, c["mp"], c["mm"], p, x)


@pytest.mark.parametrize("opname", ["DEO", "DOE", "C", "CDAG", "CCDAG"])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_partitioned_operator(case, opname, parity, prec):
    dwf = case["dwf"]
    op = getattr(dwf, "OP_" + opname)
    if op in (dwf.OP_DEO, dwf.OP_DOE) and parity == 1:
        pytest.skip("parity argument not used by this operator")
    got = dwf.dwf_part_apply(case["parts"], op, prec, parity, case["x"])
    want = _want(case, op, parity)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < TOL[prec]
    if prec in (0, 1):
        whole = dwf.dwf_apply_eo(case["whole"].h, op, prec, parity, case["x"])
        assert np.array_equal(got, whole)


def test_invalid_decompositions_and_calls(gpu_lib):
    dwf = gpu_lib
    ns = 4
    om, sg = inputs.weights("shamir", ns)
    dims = (4, 4, 4, 8)
    for grid, coord in [((1, 1, 1, 3), (0, 0, 0, 0)),    # 8 not divisible by 3
                        ((1, 1, 1, 8), (0, 0, 0, 0)),    # blocks of extent 1
                        ((1, 1, 1, 2), (0, 0, 0, 2))]:   # coordinate outside the grid
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_create_part(dims, grid, coord, ns, M0, 0.05, om, sg)
        assert e.value.status == dwf.DWF_EINVAL
    U = inputs.gauge_field(dims, 0.5, seed=53)
    parts = make_parts(dwf, dims, (1, 1, 1, 2), ns, 0.05, om, sg, U)
    x = inputs.gaussian_source(dims, ns, seed=54)
    try:
        with pytest.raises(dwf.DwfError) as e:      # a block missing
            dwf.dwf_part_apply(parts[:1], dwf.OP_C, 1, 1, x)
        assert e.value.status == dwf.DWF_EINVAL
        with pytest.raises(dwf.DwfError) as e:      # a block twice
            dwf.dwf_part_apply([parts[0], parts[0]], dwf.OP_C, 1, 1, x)
        assert e.value.status == dwf.DWF_EINVAL
        with pytest.raises(dwf.DwfError) as e:      # a part is not a whole-lattice context
            dwf.dwf_apply_eo(parts[0], dwf.OP_C, 1, 1, inputs.gaussian_source((4, 4, 4, 4), ns, seed=1))
        assert e.value.status == dwf.DWF_EINVAL
        other = dwf.dwf_create_part(dims, (1, 1, 1, 2), (0, 0, 0, 1), ns, M0, 0.1, om, sg)
        try:
            dwf.dwf_load_gauge_part(other, U)
            with pytest.raises(dwf.DwfError) as e:  # parts of different operators
                dwf.dwf_part_apply([parts[0], other], dwf.OP_C, 1, 1, x)
            assert e.value.status == dwf.DWF_EINVAL
        finally:
            dwf.dwf_destroy(other)
    finally:
        for p in parts:
            dwf.dwf_destroy(p)


@pytest.mark.parametrize("grid,system,prec", [((1, 1, 1, 2), 0, 1), ((2, 1, 2, 1), 0, 1), ((2, 2, 2, 2), 1, 1),
                                              ((1, 1, 2, 2), 0, 0), ((1, 1, 1, 2), 0, 2)])
def test_partitioned_solve(gpu_lib, grid, system, prec):
    dwf = gpu_lib
    dims, ns, mq = (4, 4, 4, 8), 8, 0.05
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=55)
    sp = 1
    rhs = inputs.gaussian_source(dims, ns, seed=56, parity=sp if system == 1 else None)
    parts = make_parts(dwf, dims, grid, ns, 0.05, om, sg, U)
    try:
        x, st = dwf.dwf_part_solve(parts, rhs, system=system, schur_parity=sp, inner_prec=prec, tol=1e-10)
    finally:
        for p in parts:
            dwf.dwf_destroy(p)
    assert st["converged"] == 1 and st["restarts"] >= 1
    if system == 0:
        res = np.linalg.norm(rhs - oracle.dfull(dims, ns, U, M0, mq, om, sg, x)) / np.linalg.norm(rhs)
        assert abs(st["true_res_full"] - res) < 1e-11
    else:
        mp, mm = oracle.m5(ns, M0, mq, om, sg)
        res = np.linalg.norm(rhs - oracle.ccdag_op(dims, ns, U, mp, mm, sp, x)) / np.linalg.norm(rhs)
    assert res <= 1e-10, f"oracle true residual {res:.3e}, stats {st}"
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as whole:
        xw, stw = dwf.dwf_solve(whole.h, rhs, system=system, schur_parity=sp, inner_prec=prec, tol=1e-10)
    assert np.linalg.norm(x - xw) / np.linalg.norm(xw) < 1e-6
