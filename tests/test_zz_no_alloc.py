"""The allocation-free operator entry point (dwf_apply_eo_dev_static), against the FP64 CPU
oracle and against dwf_apply_eo_dev.

Some callers cannot let a library allocate device memory: applications whose GPU memory is
owned by their own pool allocator (a framework's caching allocator already holding the
device) or held to a fixed budget, and paths that must not meet the device-wide
synchronisation a cudaMalloc/cudaFree can bring.  dwf_apply_eo_dev_static serves them
from a static device array inside the library.  Every operator is called through the C-ABI
on the same inputs, twice in a row (the static array keeps the previous call's contents,
so the second call checks that nothing stale leaks through), and must agree with the
oracle and with dwf_apply_eo_dev within the parity tests' tolerances: FP64 1e-12, FP32
1e-5, fp16 5e-3 (max |difference| / max |reference|).  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import pytest

import oracle
from paper_1101_0423_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}
M0, MQ = 1.8, 0.03


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1101_0423_gb300 import dwf
    dwf.load()
    dims, ns = (6, 4, 4, 6), 12        # 288 half-lattice sites: several CTA tiles, ragged tail
    om, sg = inputs.weights("cosine", ns)
    U = inputs.gauge_field(dims, 0.5, seed=41)
    ctx = dwf.Context(dims, ns, M0, MQ, om, sg, U)
    xh = [inputs.gaussian_source(dims, ns, seed=42 + k) for k in range(2)]
    xs = [torch.from_numpy(x).cuda() for x in xh]
    mp, mm = oracle.m5(ns, M0, MQ, om, sg)
    yield dwf, ctx, xs, dict(dims=dims, ns=ns, U=U, mp=mp, mm=mm, xh=xh)
    ctx.close()


def _oracle(dwf, o, op, parity, x):
    d, ns, U, mp, mm = o["dims"], o["ns"], o["U"], o["mp"], o["mm"]
    if op == dwf.OP_DEO:
        return oracle.hop(d, ns, U, 0, x)
    if op == dwf.OP_DOE:
        return oracle.hop(d, ns, U, 1, x)
    if op == dwf.OP_M5:
        return oracle.apply_s(d, ns, mp, mm, x, parity=parity)
    if op == dwf.OP_M5T:
        return oracle.apply_s(d, ns, mp, mm, x, transpose=True, parity=parity)
    if op == dwf.OP_C:
        return oracle.c_op(d, ns, U, mp, mm, parity, x)
    if op == dwf.OP_CDAG:
        return oracle.cdag_op(d, ns, U, mp, mm, parity, x)
    return oracle.ccdag_op(d, ns, U, mp, mm, parity, x)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("opname", ["DEO", "DOE", "M5", "M5T", "C", "CDAG", "CCDAG"])
@pytest.mark.parametrize("parity", [0, 1])
def test_static_variant_matches_oracle_and_allocating_entry_point(setup, opname, prec, parity):
    import torch
    dwf, ctx, xs, o = setup
    op = getattr(dwf, "OP_" + opname)
    stream = torch.cuda.current_stream()
    for x, xh in zip(xs, o["xh"]):                 # two calls in a row
        want = torch.empty_like(x)
        got = torch.full_like(x, float("nan"))     # the output is fully written by the call
        dwf.dwf_apply_eo_dev(ctx.h, op, prec, parity, x, want, stream=stream)
        dwf.dwf_apply_eo_dev_static(ctx.h, op, prec, parity, x, got, stream=stream)
        stream.synchronize()
        assert not torch.isnan(got).any()
        assert _rel(got, want) <= TOL[prec]
        ref = torch.from_numpy(_oracle(dwf, o, op, parity, xh))
        assert _rel(got.cpu(), ref) <= TOL[prec]


def test_static_variant_16bit_after_its_gauge_exists(setup):
    import torch
    dwf, ctx, xs, o = setup
    stream = torch.cuda.current_stream()
    for x in xs:
        want, got = torch.empty_like(x), torch.empty_like(x)
        dwf.dwf_apply_eo_dev(ctx.h, dwf.OP_CCDAG, dwf.PREC_F16, 1, x, want, stream=stream)
        dwf.dwf_apply_eo_dev_static(ctx.h, dwf.OP_CCDAG, dwf.PREC_F16, 1, x, got, stream=stream)
        stream.synchronize()
        assert _rel(got, want) <= TOL[2]


def test_static_variant_rejects_what_it_cannot_serve(setup):
    import torch
    dwf, ctx, xs, o = setup
    out = torch.empty_like(xs[0])
    with pytest.raises(dwf.DwfError) as e:
        dwf.dwf_apply_eo_dev_static(ctx.h, dwf.OP_DFULL, dwf.PREC_F32, 0, xs[0], out)
    assert e.value.status == dwf.DWF_EINVAL
    with pytest.raises(dwf.DwfError) as e:        # bf16 links not built on this context yet
        dwf.dwf_apply_eo_dev_static(ctx.h, dwf.OP_C, dwf.PREC_BF16, 1, xs[0], out)
    assert e.value.status == dwf.DWF_EINVAL


def test_static_variant_size_limit():
    """8^3 x 16, Ns = 20: 81,920 5D half-sites need ~79 MB of FP64 work fields (over the
    64 MiB array) but ~39 MB in FP32."""
    import torch
    from paper_1101_0423_gb300 import dwf
    dims, ns = (8, 8, 8, 16), 20
    om, sg = inputs.weights("shamir", ns)
    U = inputs.gauge_field(dims, 0.5, seed=43)
    x = torch.from_numpy(inputs.gaussian_source(dims, ns, seed=44)).cuda()
    with dwf.Context(dims, ns, 1.8, 0.05, om, sg, U) as ctx:
        out = torch.empty_like(x)
        with pytest.raises(dwf.DwfError) as e:
            dwf.dwf_apply_eo_dev_static(ctx.h, dwf.OP_CCDAG, dwf.PREC_F64, 1, x, out)
        assert e.value.status == dwf.DWF_EINVAL and "too large" in str(e.value)
        want = torch.empty_like(x)
        dwf.dwf_apply_eo_dev(ctx.h, dwf.OP_CCDAG, dwf.PREC_F32, 1, x, want)
        dwf.dwf_apply_eo_dev_static(ctx.h, dwf.OP_CCDAG, dwf.PREC_F32, 1, x, out)
        torch.cuda.synchronize()
        assert _rel(out, want) <= TOL[1]
