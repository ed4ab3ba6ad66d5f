"""Server host logic without a GPU: argument validation, admission against the memory
budget, and failure propagation when no device can run a solve.

On a machine without a GPU the server still queues and admits; the worker that picks a
request reports DWF_ECUDA through dwf_poll instead of crashing or hanging.  (On a GPU
machine that last case is covered by the GPU tests instead.)
"""
import time

import numpy as np
import pytest

from paper_1101_0423_gb300 import inputs


@pytest.fixture(scope="module")
def dwf():
    from paper_1101_0423_gb300 import build, dwf
    build.build()
    dwf.load()
    return dwf


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


DIMS, NS = (4, 4, 4, 4), 4


def _req_args():
    om, sg = inputs.weights("shamir", NS)
    return om, sg, inputs.gaussian_source(DIMS, NS, seed=5)


def test_malformed_requests_are_rejected(dwf):
    srv = dwf.dwf_server_create(hbm_budget_gb=1.0, max_inflight=2)
    try:
        g = dwf.dwf_server_add_gauge(srv, DIMS, inputs.unit_gauge(DIMS))
        om, sg, rhs = _req_args()
        bad = [dict(Ns=0), dict(m0=2.5), dict(gauge=7), dict(dims=(4, 4, 4, 8)), dict(omega=-np.ones(NS)),
               dict(system=5), dict(inner_prec=9)]
        for b in bad:
            kw = dict(dims=DIMS, Ns=NS, m0=1.8, mq=0.05, omega=om, sigma=sg, gauge=g, rhs=rhs)
            extra = {k: v for k, v in b.items() if k in ("system", "inner_prec")}
            kw.update({k: v for k, v in b.items() if k not in extra})
            if kw["Ns"] != NS:
                kw["omega"], kw["sigma"] = np.ones(max(kw["Ns"], 1)), np.zeros(max(kw["Ns"], 1))
            with pytest.raises(dwf.DwfError) as e:
                dwf.dwf_submit(srv, **kw, **extra)
            assert e.value.status == dwf.DWF_EINVAL, b
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_server_add_gauge(srv, (3, 4, 4, 4), inputs.unit_gauge((4, 4, 4, 4)))
        assert e.value.status == dwf.DWF_EINVAL
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_poll(srv, 12345)
        assert e.value.status == dwf.DWF_EINVAL
    finally:
        dwf.dwf_server_destroy(srv)


def test_request_larger_than_budget_is_refused(dwf):
    srv = dwf.dwf_server_create(hbm_budget_gb=1e-4, max_inflight=1)   # ~100 KiB
    try:
        g = dwf.dwf_server_add_gauge(srv, DIMS, inputs.unit_gauge(DIMS))
        om, sg, rhs = _req_args()
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_submit(srv, DIMS, NS, 1.8, 0.05, om, sg, g, rhs)
        assert e.value.status == dwf.DWF_ENOMEM
        assert dwf.dwf_server_get_stats(srv)["submitted"] == 0
    finally:
        dwf.dwf_server_destroy(srv)


@pytest.mark.skipif(has_gpu(), reason="exercises the no-device path")
def test_without_device_the_failure_reaches_poll(dwf):
    srv = dwf.dwf_server_create(hbm_budget_gb=2.0, max_inflight=2)
    try:
        g = dwf.dwf_server_add_gauge(srv, DIMS, inputs.unit_gauge(DIMS))
        om, sg, rhs = _req_args()
        tickets = [dwf.dwf_submit(srv, DIMS, NS, 1.8, 0.05, om, sg, g, rhs) for _ in range(3)]
        done = {}
        t0 = time.time()
        while len(done) < 3 and time.time() - t0 < 30:
            for t in tickets:
                if t not in done:
                    r = dwf.dwf_poll(srv, t)
                    if r is not None:
                        done[t] = r[1]
            time.sleep(0.01)
        assert len(done) == 3
        assert all(r["status"] == dwf.DWF_ECUDA for r in done.values())
        st = dwf.dwf_server_get_stats(srv)
        assert st["completed"] == 3 and st["in_flight"] == 0 and st["hbm_reserved_gb"] == 0
    finally:
        dwf.dwf_server_destroy(srv)


def _wait(dwf, srv, tickets, timeout=60):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in done:
                r = dwf.dwf_poll(srv, t)
                if r is not None:
                    done[t] = r[1]
        time.sleep(0.01)
    return done


def test_cancel_withdraws_a_queued_request(dwf):
    """With admission closed, requests queue; a queued one can be withdrawn (its ticket is
    gone), the others run once admission opens, and a finished one can no longer be
    withdrawn.  Host logic only: without a GPU the admitted solves end with DWF_ECUDA."""
    srv = dwf.dwf_server_create(hbm_budget_gb=2.0, max_inflight=2)
    try:
        g = dwf.dwf_server_add_gauge(srv, DIMS, inputs.unit_gauge(DIMS))
        om, sg, rhs = _req_args()
        dwf.dwf_server_set_admission(srv, False)
        t = [dwf.dwf_submit(srv, DIMS, NS, 1.8, 0.05, om, sg, g, rhs) for _ in range(3)]
        time.sleep(0.05)
        st = dwf.dwf_server_get_stats(srv)
        assert st["queued"] == 3 and st["in_flight"] == 0 and st["completed"] == 0
        assert dwf.dwf_cancel(srv, t[1]) is True
        for call in (lambda: dwf.dwf_cancel(srv, t[1]), lambda: dwf.dwf_poll(srv, t[1])):
            with pytest.raises(dwf.DwfError) as e:
                call()
            assert e.value.status == dwf.DWF_EINVAL
        st = dwf.dwf_server_get_stats(srv)
        assert st["queued"] == 2 and st["cancelled"] == 1 and st["submitted"] == 3
        dwf.dwf_server_set_admission(srv, True)
        t0 = time.time()
        while dwf.dwf_server_get_stats(srv)["completed"] < 2 and time.time() - t0 < 60:
            time.sleep(0.01)
        assert dwf.dwf_cancel(srv, t[0]) is False  # finished, not yet collected
        done = _wait(dwf, srv, [t[0], t[2]])
        assert len(done) == 2
        want = dwf.DWF_OK if has_gpu() else dwf.DWF_ECUDA
        assert all(r["status"] == want for r in done.values())
        st = dwf.dwf_server_get_stats(srv)
        assert st["completed"] == 2 and st["queued"] == 0 and st["cancelled"] == 1
    finally:
        dwf.dwf_server_destroy(srv)


def test_cancel_rejects_unknown_tickets_and_null_servers(dwf):
    srv = dwf.dwf_server_create(hbm_budget_gb=1.0, max_inflight=1)
    try:
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_cancel(srv, 999)
        assert e.value.status == dwf.DWF_EINVAL
    finally:
        dwf.dwf_server_destroy(srv)
    assert dwf.load().dwf_cancel(None, 1) == dwf.DWF_EINVAL
    assert dwf.load().dwf_server_set_admission(None, 1) == dwf.DWF_EINVAL
