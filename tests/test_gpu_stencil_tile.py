"""One-system FP32 stencil passes with the links staged in shared memory by
bulk asynchronous copies (lattices whose x0-x1 planes are whole tiles of 256
sites).

The staged kernel (opt-in: MSC_STAG_TILE=1 for a context) sums in the same
order as the direct one, so a solve with staging must reproduce the direct
solve bit for bit, and both must match the FP64 oracle (true residual <=
1e-10 per shift, x_s within 1e-8).

The copies complete on an mbarrier whose wait is bounded in time. With
MSC_TEST_NO_COPY=1 the kernel issues no copies, so nothing completes the
barrier and every wait runs out (after MSC_WAIT_NS = 1 ms): the solve must
return MSC_ERR_TIMEOUT, and a new context must solve normally afterwards.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402


def _ctx(env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return msc.msc_create(0, torch.cuda.current_stream())
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module", autouse=True)
def lib():
    msc.load()


@pytest.mark.parametrize("dims,nc", [((16, 16, 16, 16), 3), ((32, 8, 6, 4), 3), ((16, 16, 4, 6), 2)])
def test_staged_solve_equals_unstaged_and_oracle(dims, nc):
    p = inputs.staggered_problem(dims, nc, 0.08, 0.7, inputs.log_shifts(1e-3, 2.0, 6), 1, 1e-10, 7300)
    xs = []
    for env in ({"MSC_STAG_TILE": "1"}, {}):
        c = _ctx(env)
        op = msc.msc_op_staggered(c, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
        x, info = msc.solve(c, op, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol)
        assert info.status == 0
        xs.append(x.cpu().numpy())
        msc.msc_op_destroy(op)
        msc.msc_destroy(c)
    assert np.array_equal(xs[0], xs[1])
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-13)
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, xs[0][0])
    assert np.all(rho <= p.tol), rho
    for s in range(len(p.sigma)):
        err = np.linalg.norm(xs[0][0, s] - ref.x[s]) / np.linalg.norm(ref.x[s])
        assert err <= 1e-8, (s, err)


def test_wait_that_runs_out_reports_timeout():
    p = inputs.staggered_problem((16, 16, 16, 16), 3, 0.1, 0.6, [0.01, 0.1], 1, 1e-10, 7400)
    c = _ctx({"MSC_STAG_TILE": "1", "MSC_TEST_NO_COPY": "1", "MSC_WAIT_NS": "1000000"})
    op = msc.msc_op_staggered(c, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    with pytest.raises(msc.MscError) as e:
        msc.solve(c, op, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol)
    assert e.value.code == msc.MSC_ERR_TIMEOUT
    # the FP32 operator apply runs the same staged pass and reports it too
    v = torch.from_numpy(p.b[0]).cuda()
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_apply(c, op, 0.0, v, torch.empty_like(v), msc.MSC_FP32)
    assert e.value.code == msc.MSC_ERR_TIMEOUT
    msc.msc_op_destroy(op)
    msc.msc_destroy(c)
    torch.cuda.synchronize()
    c = _ctx({})
    op = msc.msc_op_staggered(c, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    x, info = msc.solve(c, op, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol)
    assert info.status == 0 and np.all(info.true_rel_resid <= p.tol)
    msc.msc_op_destroy(op)
    msc.msc_destroy(c)
