"""GPU parity of the multi-shift BiCGStab (BiCGStab-M) for non-Hermitian
shifted families, through the C ABI, against the FP64 oracle's BiCGStab-M
(its recurrences pinned by dense solves and by CG-M on the normal equations).

Tolerances: x_s within 1e-8 relative of the oracle's solution (solved to
1e-13), and the FP64 true residual |b - (A + sigma_s) x_s| <= tol |b| for
every shift, recomputed by the oracle from the returned x_s.
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def ctx():
    msc.load()
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


@pytest.mark.parametrize("nbr,bd", [(37, 1), (70, 2), (45, 3)])
def test_random_nonhermitian_bsr_ragged(ctx, nbr, bd):
    rp, ci, va, A = inputs.random_nonhermitian_bsr(nbr, bd, 5, 0.5, 0.3, 90 + bd)
    n = A.shape[0]
    b = inputs.gaussian_source(n, 91)
    sig = np.array([-0.05, 0.0, 0.02, 0.3, 1.5, 6.0])       # any finite shifts
    op = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    x, info = msc.solve_nonherm(ctx, op, b, sig, tol=1e-10)
    assert info.status == 0
    ref = oracle.bicgstabm_bsr(rp, ci, va, b, sig, 1e-13)
    assert ref.status == 0
    for s, sv in enumerate(sig):
        xd = np.linalg.solve(A + sv * np.eye(n), b)
        assert rel(x[s], xd) <= 1e-8, (s, rel(x[s], xd))
        assert rel(x[s], ref.x[s]) <= 1e-8, (s, rel(x[s], ref.x[s]))
        r = b - oracle.bsr_apply(rp, ci, va, x[s], sigma=sv)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
        assert info.true_rel_resid[0, s] <= 1e-10
    msc.msc_op_destroy(op)


def test_staggered_dirac_multimass_against_oracle(ctx):
    """The multi-mass family (m + sigma_s + D) x_s = b of the staggered Dirac
    operator, 8^4 SU(3), m = 0.05, 8 masses, given to the library as
    block-CSR (9 blocks per row); right-hand sides on the host and on the
    device."""
    dims, nc, m = (8, 8, 8, 8), 3, 0.05
    U = inputs.su_n_links(dims, nc, 0.6, 95)
    rp, ci, va = inputs.staggered_dirac_bsr(U, dims, nc, m)
    n = inputs.volume(dims) * nc
    b = inputs.gaussian_source(n, 96, nrhs=2)
    sig = inputs.log_shifts(1e-3, 1.0, 8)
    op = msc.msc_op_bsr(ctx, inputs.volume(dims), nc, rp, ci, va)
    x_host, info = msc.solve_nonherm(ctx, op, b, sig, tol=1e-10)
    x_dev, info_d = msc.solve_nonherm(ctx, op, torch.from_numpy(b).cuda(), sig, tol=1e-10)
    assert info.status == 0 and info_d.status == 0
    assert np.array_equal(x_host, x_dev.cpu().numpy())
    for r in range(2):
        ref = oracle.bicgstabm_dirac(U, dims, nc, m + sig[0], b[r], sig - sig[0], 1e-13)
        assert ref.status == 0
        for s in range(len(sig)):
            assert rel(x_host[r, s], ref.x[s]) <= 1e-8, (r, s)
            res = b[r] - oracle.dirac_apply(U, dims, nc, m, x_host[r, s], sigma=sig[s])
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(b[r])
    assert np.all(info.shift_iters >= 1)
    msc.msc_op_destroy(op)


def test_nonherm_edges(ctx):
    rp, ci, va, A = inputs.random_nonhermitian_bsr(20, 2, 3, 0.5, 0.3, 97)
    op = msc.msc_op_bsr(ctx, 20, 2, rp, ci, va)
    x, info = msc.solve_nonherm(ctx, op, np.zeros(40, np.complex128), [0.1, 1.0])
    assert info.status == 0 and info.iters == 0 and np.all(x == 0)
    # one shift, and the cap
    b = inputs.gaussian_source(40, 98)
    x, info = msc.solve_nonherm(ctx, op, b, [0.25])
    assert np.linalg.norm(b - (A @ x[0] + 0.25 * x[0])) <= 1e-10 * np.linalg.norm(b)
    x, info = msc.solve_nonherm(ctx, op, b, [0.0, 1.0], max_iter=2, raise_on_error=False)
    assert info.status == msc.MSC_ERR_NOT_CONVERGED and info.iters == 2
    x, info = msc.solve_nonherm(ctx, op, b, [0.5], max_iter=0, raise_on_error=False)
    assert info.status == msc.MSC_ERR_NOT_CONVERGED and info.iters == 0 and np.all(x == 0)
    # what the solver does not take
    p = inputs.lattice_4x4_su3_8shifts()
    sop = msc.msc_op_staggered(ctx, p.nc, p.dims, p.links, p.mass)
    with pytest.raises(msc.MscError) as e:
        msc.solve_nonherm(ctx, sop, p.b[0], p.sigma)
    assert e.value.code == msc.MSC_ERR_UNSUPPORTED
    with pytest.raises(msc.MscError) as e:
        msc.solve_nonherm(ctx, op, b, [np.inf])
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(sop)
    msc.msc_op_destroy(op)


def test_breakdown_is_reported(ctx):
    """A real skew-symmetric A and a real b: b^T A b = 0, so the first
    denominator (r~, A p) of BiCGStab vanishes; the solve reports it."""
    nbr = 16
    rp, ci, va = [0], [], []
    for i in range(nbr):
        if i > 0:
            ci.append(i - 1); va.append(-1.0)
        if i < nbr - 1:
            ci.append(i + 1); va.append(1.0)
        rp.append(len(ci))
    rp, ci = np.asarray(rp, np.int64), np.asarray(ci, np.int32)
    va = np.asarray(va, np.complex128).reshape(-1, 1, 1)
    b = np.arange(1, nbr + 1, dtype=np.float64).astype(np.complex128)
    assert oracle.bicgstabm_bsr(rp, ci, va, b, [0.0], 1e-10).status == 7
    op = msc.msc_op_bsr(ctx, nbr, 1, rp, ci, va)
    with pytest.raises(msc.MscError) as e:
        msc.solve_nonherm(ctx, op, b, [0.0])
    assert e.value.code == msc.MSC_ERR_BREAKDOWN
    # the context stays usable
    x, info = msc.solve_nonherm(ctx, op, b, [2.0])
    assert info.status == 0
    msc.msc_op_destroy(op)
