"""msc_op_apply_noalloc: the staggered operator apply for callers that may not
let a library allocate device memory (code under another framework's memory
pool or allocator, latency-bound loops where cudaMalloc may block or fail).

Its result must equal the oracle's FP64 (A + sigma) x and msc_op_apply's
(which stages vectors in a workspace it allocates), both to the FP64 operator
tolerance of the other GPU tests, 1e-13 relative, on two calls in a row: the
second call reuses the fixed scratch array the first one left behind.
Collected last so that a failure here does not hide the rest of the suite; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402

TOL = 1e-13


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    msc.load()
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


@pytest.mark.parametrize("nc,dims,sigma", [(3, (8, 8, 8, 8), 0.25), (2, (6, 4, 4, 8), 0.0)])
def test_noalloc_apply_equals_allocating_apply(ctx, nc, dims, sigma):
    U = inputs.su_n_links(dims, nc, 0.7, 900 + nc)
    op = msc.msc_op_staggered(ctx, nc, dims, torch.from_numpy(U).cuda(), 0.1)
    n = inputs.volume(dims) * nc
    stream = torch.cuda.current_stream()
    for call in range(2):
        x = torch.from_numpy(inputs.gaussian_source(n, 910 + call)).cuda()
        ref = torch.empty_like(x)
        msc.msc_op_apply(ctx, op, sigma, x, ref, msc.MSC_FP64)
        out = torch.full_like(x, float("nan"))
        msc.msc_op_apply_noalloc(op, sigma, x, out, stream)
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL, (call, rel(out, ref))
        want = oracle.staggered_apply(U, dims, nc, 0.1, x.cpu().numpy(), sigma)
        got = out.cpu().numpy()
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= TOL, (call, err)
    msc.msc_op_destroy(op)


def test_noalloc_apply_allocates_nothing_and_rejects_oversize(ctx):
    dims, nc = (8, 8, 8, 8), 3
    U = inputs.su_n_links(dims, nc, 0.5, 920)
    op = msc.msc_op_staggered(ctx, nc, dims, torch.from_numpy(U).cuda(), 0.2)
    n = inputs.volume(dims) * nc
    x = torch.from_numpy(inputs.gaussian_source(n, 921)).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    msc.msc_op_apply_noalloc(op, 0.1, x, out, stream)  # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        msc.msc_op_apply_noalloc(op, 0.1, x, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # out may equal in
    ref = torch.empty_like(x)
    msc.msc_op_apply(ctx, op, 0.1, x, ref, msc.MSC_FP64)
    y = x.clone()
    msc.msc_op_apply_noalloc(op, 0.1, y, y, stream)
    torch.cuda.synchronize()
    assert rel(y, ref) <= TOL
    # host pointers are refused (nothing is staged)
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_apply_noalloc(op, 0.1, x.cpu().numpy(), out, stream)
    assert e.value.code == msc.MSC_ERR_ARG
    # the binding refuses a tensor of the wrong type or length before the call
    with pytest.raises(ValueError):
        msc.msc_op_apply_noalloc(op, 0.1, x.to(torch.complex64), out, stream)
    with pytest.raises(ValueError):
        msc.msc_op_apply_noalloc(op, 0.1, x[:-1], out[:-1], stream)
    msc.msc_op_destroy(op)
    # more than 2^20 complex unknowns does not fit the fixed array
    big = (32, 32, 32, 12)
    Ub = inputs.su_n_links(big, 3, 0.0, 0)
    opb = msc.msc_op_staggered(ctx, 3, big, torch.from_numpy(Ub).cuda(), 0.1)
    nb = inputs.volume(big) * 3
    assert nb > 1 << 20
    xb = torch.zeros(nb, dtype=torch.complex128, device="cuda")
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_apply_noalloc(opb, 0.0, xb, xb, stream)
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(opb)
