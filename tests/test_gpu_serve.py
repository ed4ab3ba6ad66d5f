"""Served solves (dwf_submit / dwf_poll) on the GPU.

Requests of different lattices, Ns, masses, weight sets, systems and inner precisions are
submitted together and overlap on the device; every result must be identical (bit for
bit: the reductions have a fixed order) to the same solve run alone through dwf_solve, and
the oracle must confirm the true residual.  A tight memory budget must serialise the
solves without changing any result.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
M0 = 1.8

# (dims, Ns, weights, mq, system, schur_parity, inner precision, gauge seed)
CASES = [
    ((4, 4, 4, 4), 8, "shamir", 0.05, 1, 0, 1, 1),
    ((4, 4, 4, 4), 8, "cosine", 0.02, 0, 1, 1, 1),
    ((6, 4, 4, 6), 12, "borici", 0.1, 0, 1, 3, 2),
    ((8, 8, 8, 8), 8, "cosine", 0.05, 0, 1, 1, 3),
    ((4, 4, 4, 4), 4, "shamir", 0.005, 0, 0, 2, 1),
]


def run_all(dwf, srv, gauges, cases, seeds):
    tickets = []
    for (dims, ns, kind, mq, system, sp, prec, gseed), seed in zip(cases, seeds):
        om, sg = inputs.weights(kind, ns)
        rhs = inputs.gaussian_source(dims, ns, seed=seed, parity=sp if system == 1 else None)
        tickets.append(dwf.dwf_submit(srv, dims, ns, M0, mq, om, sg, gauges[(dims, gseed)], rhs,
                                      system=system, schur_parity=sp, inner_prec=prec, tol=1e-10))
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < 600:
        for i, t in enumerate(tickets):
            if i in out:
                continue
            buf = np.empty(int(np.prod(cases[i][0])) * cases[i][1] * 24)
            r = dwf.dwf_poll(srv, t, buf)
            if r is not None:
                out[i] = (buf, r[1])
        time.sleep(0.005)
    assert len(out) == len(tickets), "requests did not finish"
    return [out[i] for i in range(len(tickets))]


def solve_alone(dwf, case, seed):
    dims, ns, kind, mq, system, sp, prec, gseed = case
    om, sg = inputs.weights(kind, ns)
    U = inputs.gauge_field(dims, 0.5, seed=gseed)
    rhs = inputs.gaussian_source(dims, ns, seed=seed, parity=sp if system == 1 else None)
    with dwf.Context(dims, ns, M0, mq, om, sg, U) as ctx:
        x, st = dwf.dwf_solve(ctx.h, rhs, system=system, schur_parity=sp, inner_prec=prec, tol=1e-10)
    return x, rhs, U, om, sg


@pytest.fixture(scope="module")
def served(gpu_lib):
    dwf = gpu_lib
    srv = dwf.dwf_server_create(hbm_budget_gb=20.0, max_inflight=3)
    gauges = {}
    for dims, *_r, gseed in CASES:
        if (dims, gseed) not in gauges:
            gauges[(dims, gseed)] = dwf.dwf_server_add_gauge(srv, dims, inputs.gauge_field(dims, 0.5, seed=gseed))
    # two rounds of every case, interleaved, so solves of different shapes overlap
    cases = CASES + CASES
    seeds = [100 + i for i in range(len(CASES))] * 2
    results = run_all(dwf, srv, gauges, cases, seeds)
    stats = dwf.dwf_server_get_stats(srv)
    yield dwf, srv, gauges, results, stats
    dwf.dwf_server_destroy(srv)


def test_each_result_is_the_same_alone_and_in_the_mix(served):
    dwf, srv, gauges, results, stats = served
    for i, case in enumerate(CASES):
        alone, rhs, U, om, sg = solve_alone(dwf, case, 100 + i)
        for k in (i, i + len(CASES)):
            x, res = results[k]
            assert res["status"] == dwf.DWF_OK and res["stats"]["converged"] == 1
            assert np.array_equal(x, alone), f"case {i} differs in the mix"


def test_served_solutions_meet_the_residual(served):
    dwf, srv, gauges, results, stats = served
    for i, (dims, ns, kind, mq, system, sp, prec, gseed) in enumerate(CASES):
        x, res = results[i]
        om, sg = inputs.weights(kind, ns)
        U = inputs.gauge_field(dims, 0.5, seed=gseed)
        rhs = inputs.gaussian_source(dims, ns, seed=100 + i, parity=sp if system == 1 else None)
        if system == 0:
            r = rhs - oracle.dfull(dims, ns, U, M0, mq, om, sg, x)
        else:
            mp, mm = oracle.m5(ns, M0, mq, om, sg)
            r = rhs - oracle.ccdag_op(dims, ns, U, mp, mm, sp, x)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-10


def test_server_statistics(served):
    dwf, srv, gauges, results, stats = served
    assert stats["submitted"] == stats["completed"] == 2 * len(CASES)
    assert stats["in_flight"] == 0 and stats["queued"] == 0
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert stats["solves_per_s"] > 0
    assert all(r[1]["latency_ms"] >= r[1]["queue_ms"] >= 0 for r in results)


def test_requests_of_one_operator_share_a_batch(gpu_lib):
    """Requests of the same operator and settings queued together run as rows of one batched
    solve; every row's result is bit for bit the solve of that right-hand side alone."""
    dwf = gpu_lib
    srv = dwf.dwf_server_create(hbm_budget_gb=20.0, max_inflight=1)
    try:
        case = CASES[3]
        dims, ns, kind, mq, system, sp, prec, gseed = case
        g = {(dims, gseed): dwf.dwf_server_add_gauge(srv, dims, inputs.gauge_field(dims, 0.5, seed=gseed))}
        dwf.dwf_server_set_admission(srv, False)   # queue them all before any is admitted
        seeds = [300 + i for i in range(5)]
        tickets = []
        for seed in seeds:
            om, sg = inputs.weights(kind, ns)
            rhs = inputs.gaussian_source(dims, ns, seed=seed)
            tickets.append(dwf.dwf_submit(srv, dims, ns, M0, mq, om, sg, g[(dims, gseed)], rhs,
                                          system=system, schur_parity=sp, inner_prec=prec, tol=1e-10))
        dwf.dwf_server_set_admission(srv, True)
        out = []
        for t in tickets:
            buf = np.empty(int(np.prod(dims)) * ns * 24)
            while dwf.dwf_poll(srv, t, buf) is None:
                time.sleep(0.005)
            out.append(buf)
        assert dwf.dwf_server_get_stats(srv)["batched"] == len(seeds)
        for seed, x in zip(seeds, out):
            alone = solve_alone(dwf, case, seed)[0]
            assert np.array_equal(x, alone)
    finally:
        dwf.dwf_server_destroy(srv)


def test_tight_budget_serialises_without_changing_results(gpu_lib):
    """A budget that fits one small solve at a time: all finish, results unchanged."""
    dwf = gpu_lib
    srv = dwf.dwf_server_create(hbm_budget_gb=0.025, max_inflight=4)
    try:
        case = CASES[1]
        dims, ns, kind, mq, system, sp, prec, gseed = case
        g = {(dims, gseed): dwf.dwf_server_add_gauge(srv, dims, inputs.gauge_field(dims, 0.5, seed=gseed))}
        results = run_all(dwf, srv, g, [case] * 4, [100 + 1] * 4)
        alone = solve_alone(dwf, case, 101)[0]
        for x, res in results:
            assert res["status"] == dwf.DWF_OK and np.array_equal(x, alone)
        assert dwf.dwf_server_get_stats(srv)["hbm_reserved_gb"] <= 0.025
    finally:
        dwf.dwf_server_destroy(srv)
