"""Different right-hand side per shift (Sec. 5, eq. linprobgen) in polynomial
form, b_s = q_s(A) b: msc_solve_poly_rhs against the oracle, which forms each
b_s by Horner's rule and solves every shift on its own by textbook CG.

Tolerance: both solutions have FP64 true residuals rho <= 1e-10 relative to
|b_s|; A = m^2 + D^dag D with |D| <= 4, so |x - x*| / |x*| <= kappa_s (rho +
rho*), kappa_s = (m^2 + 16 + sigma_s) / (m^2 + sigma_s), and the mixed-form
target |x - x*| / |x*| <= 1e-8 is checked as well.
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    msc.load()
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


def _coefs(S, deg, seed):
    return inputs.rng(seed).uniform(-1.0, 1.0, size=(S, deg + 1))


def _check(p, x, info, coef, tol=1e-10):
    xr, bs = oracle.solve_poly_rhs_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, coef, 1e-13)
    for s in range(len(p.sigma)):
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, bs[s], p.sigma[s:s + 1],
                                             x[s][None, :])[0]
        assert rho <= tol, (s, rho)
        assert abs(rho - info.true_rel_resid[s]) <= 1e-3 * tol, (s, rho, info.true_rel_resid[s])
        err = np.linalg.norm(x[s] - xr[s]) / np.linalg.norm(xr[s])
        kap = (p.mass ** 2 + 16 + p.sigma[s]) / (p.mass ** 2 + p.sigma[s])
        rho_r = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, bs[s], p.sigma[s:s + 1],
                                               xr[s][None, :])[0]
        assert err <= kap * (rho + rho_r), (s, err)
        assert err <= 1e-8, (s, err)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("deg", [0, 1, 3])
def test_poly_rhs_4x4_matches_oracle(ctx, prec, deg):
    p = inputs.lattice_4x4_su3_8shifts()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    coef = _coefs(len(p.sigma), deg, 100 + deg)
    x, info = msc.solve_poly_rhs(ctx, op, torch.from_numpy(p.b[0]).cuda(), p.sigma, coef, tol=p.tol,
                                 precision=msc.MSC_FP64 if prec == "fp64" else msc.MSC_MIXED)
    assert info.status == 0
    _check(p, x.cpu().numpy(), info, coef)
    msc.msc_op_destroy(op)


def test_poly_rhs_ragged_lattice_and_block_csr(ctx):
    """A ragged 8x6x4x6 SU(2) lattice (sites not a multiple of a block) on the
    stencil path, then the same operator exported as block-CSR."""
    p = inputs.staggered_problem((8, 6, 4, 6), 2, 0.15, 0.6, inputs.log_shifts(1e-3, 2.0, 5), 1, 1e-10, 7000)
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    coef = _coefs(len(p.sigma), 2, 110)
    b = torch.from_numpy(p.b[0]).cuda()
    x, info = msc.solve_poly_rhs(ctx, op, b, p.sigma, coef, tol=p.tol)
    assert info.status == 0
    _check(p, x.cpu().numpy(), info, coef)
    nbr, nnzb, bd = msc.msc_op_bsr_size(op)
    rp = torch.empty(nbr + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(nnzb, dtype=torch.int32, device="cuda")
    va = torch.empty((nnzb, bd, bd), dtype=torch.complex128, device="cuda")
    msc.msc_staggered_export_bsr(ctx, op, rp, ci, va)
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    x2, info2 = msc.solve_poly_rhs(ctx, bop, b, p.sigma, coef, tol=p.tol)
    assert info2.status == 0
    _check(p, x2.cpu().numpy(), info2, coef)
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(op)


def test_poly_rhs_zero_rhs_and_root_at_minus_sigma(ctx):
    """q_s = 0 gives x_s = 0 exactly; q_s(t) = t + sigma_s (a root at
    -sigma_s, so the CG-M part vanishes) gives x_s = b exactly up to
    rounding; the other shifts are unaffected."""
    p = inputs.lattice_4x4_su3_8shifts()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    S = len(p.sigma)
    coef = _coefs(S, 1, 120)
    coef[0] = 0.0
    coef[1] = [p.sigma[1], 1.0]
    x, info = msc.solve_poly_rhs(ctx, op, p.b[0], p.sigma, coef, tol=p.tol)
    assert info.status == 0
    assert np.all(x[0] == 0)
    assert np.linalg.norm(x[1] - p.b[0]) <= 1e-12 * np.linalg.norm(p.b[0])
    xr, _ = oracle.solve_poly_rhs_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma[2:], coef[2:], 1e-13)
    for s in range(2, S):
        assert np.linalg.norm(x[s] - xr[s - 2]) <= 1e-8 * np.linalg.norm(xr[s - 2])
    msc.msc_op_destroy(op)


def test_poly_rhs_argument_errors(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    coef = _coefs(len(p.sigma), 1, 130)
    coef[2, 0] = np.nan
    with pytest.raises(msc.MscError) as e:
        msc.solve_poly_rhs(ctx, op, p.b[0], p.sigma, coef)
    assert e.value.code == msc.MSC_ERR_ARG
    with pytest.raises(msc.MscError) as e:
        msc.solve_poly_rhs(ctx, op, p.b[0], p.sigma, np.ones((len(p.sigma), 40)))
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(op)
