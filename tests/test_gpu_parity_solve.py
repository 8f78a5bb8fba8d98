"""Single-parity solve (msc_solve_parity): a source on the sites of one
parity needs only the reduced operator m^2 - D_{p,1-p} D_{1-p,p} on half the
unknowns, because A = m^2 - D^2 couples no even site to an odd one.

Oracle: the full-lattice FP64 CG-M of the embedded source (zero on the other
parity), whose solution is exactly zero on the other parity (a CPU pin); the
library's half-length x_s must equal its parity-p part. Tolerances as in the
other solve tests: FP64 true residual <= 1e-10 for every shift, x_s error
within kappa_s (rho + rho*) and <= 1e-8.
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


def _parity_sites(dims, par):
    V = inputs.volume(dims)
    x = np.arange(V)
    c = [x % dims[0], (x // dims[0]) % dims[1], (x // (dims[0] * dims[1])) % dims[2],
         x // (dims[0] * dims[1] * dims[2])]
    return np.nonzero(((c[0] + c[1] + c[2] + c[3]) & 1) == par)[0]


def _embed(bc, sites, V, nc):
    full = np.zeros((V, nc), dtype=np.complex128)
    full[sites] = bc.reshape(-1, nc)
    return full.reshape(-1)


def _run(ctx, p, par, prec, nrhs=1):
    V = inputs.volume(p.dims)
    sites = _parity_sites(p.dims, par)
    g = inputs.rng(8000 + par)
    bc = (g.standard_normal((nrhs, len(sites) * p.nc)) + 1j * g.standard_normal((nrhs, len(sites) * p.nc)))
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    x, info = msc.solve_parity(ctx, op, par, torch.from_numpy(bc).cuda(), p.sigma, tol=p.tol, precision=prec)
    assert info.status == 0
    x = x.cpu().numpy()
    for r in range(nrhs):
        bf = _embed(bc[r], sites, V, p.nc)
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, bf, p.sigma, 1e-13)
        assert ref.status == 0
        for s in range(len(p.sigma)):
            xf = _embed(x[r, s], sites, V, p.nc)
            rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, bf, p.sigma[s:s + 1],
                                                 xf[None, :])[0]
            assert rho <= p.tol, (r, s, rho)
            assert abs(rho - info.true_rel_resid[r, s]) <= 1e-3 * p.tol
            rho_r = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, bf, p.sigma[s:s + 1],
                                                   ref.x[s][None, :])[0]
            want = ref.x[s].reshape(V, p.nc)[sites].reshape(-1)
            err = np.linalg.norm(x[r, s] - want) / np.linalg.norm(want)
            kap = (p.mass ** 2 + 16 + p.sigma[s]) / (p.mass ** 2 + p.sigma[s])
            assert err <= kap * (rho + rho_r) and err <= 1e-8, (r, s, err)
    msc.msc_op_destroy(op)
    return info


@pytest.mark.parametrize("par", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parity_solve_4x4_matches_oracle(ctx, par, prec):
    p = inputs.lattice_4x4_su3_8shifts()
    _run(ctx, p, par, msc.MSC_FP64 if prec == "fp64" else msc.MSC_MIXED)


def test_parity_solve_ragged_su2_three_rhs(ctx):
    """An 8x6x4x10 SU(2) lattice (half volume 960 sites, several blocks and a
    ragged tail) with three right-hand sides through the grouped passes."""
    p = inputs.staggered_problem((8, 6, 4, 10), 2, 0.1, 0.7, inputs.log_shifts(1e-3, 1.0, 6), 1, 1e-10, 7100)
    _run(ctx, p, 1, msc.MSC_MIXED, nrhs=3)


def test_parity_solve_equals_full_solve_on_embedded_source(ctx):
    """Same 8^4 source through msc_solve (embedded) and msc_solve_parity:
    the same solution on the parity's sites, fewer bytes, zero elsewhere."""
    p = inputs.lattice_32x4_su3_20shifts(L=8, nrhs=1)
    V = inputs.volume(p.dims)
    sites = _parity_sites(p.dims, 0)
    bc = p.b[0].reshape(V, p.nc)[sites].reshape(-1)
    bf = _embed(bc, sites, V, p.nc)
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    xf, infof = msc.solve(ctx, op, bf, p.sigma, tol=p.tol)
    xh, infoh = msc.solve_parity(ctx, op, 0, bc, p.sigma, tol=p.tol)
    assert infof.status == 0 and infoh.status == 0
    for s in range(len(p.sigma)):
        full = xf[s].reshape(V, p.nc)
        want = full[sites].reshape(-1)
        assert np.linalg.norm(xh[s] - want) <= 1e-8 * np.linalg.norm(want)
    msc.msc_op_destroy(op)


def test_parity_argument_errors(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    bc = np.ones(inputs.volume(p.dims) // 2 * p.nc, dtype=np.complex128)
    with pytest.raises(msc.MscError) as e:
        msc.solve_parity(ctx, op, 2, bc, p.sigma)
    assert e.value.code == msc.MSC_ERR_ARG
    rp, ci, va, _ = inputs.random_hpd_bsr(8, 1, 2, 1.0, 90)
    bop = msc.msc_op_bsr(ctx, 8, 1, rp, ci, va)
    with pytest.raises(msc.MscError) as e:
        msc.solve_parity(ctx, bop, 0, np.ones(4, dtype=np.complex128), p.sigma)
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(op)
