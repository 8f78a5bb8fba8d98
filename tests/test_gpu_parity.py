"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Tolerances:
  * FP64 operator kernels: 1e-13 relative (rounding order only);
  * FP32 operator kernels: 2e-6 relative (FP32 data and arithmetic; a 3x3
    complex product over 8 neighbours accumulates a few units of 2^-24);
  * solves: true relative residual <= tol = 1e-10 in FP64 for every shift,
    and x_s within 1e-8 relative of the oracle's solution (solved to 1e-13).
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
    assert torch.cuda.is_available()
    msc.load()
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


def stag_op(ctx, p_links, dims, nc, mass, flags=0, device=True):
    links = torch.from_numpy(p_links).cuda() if device else np.ascontiguousarray(p_links)
    return msc.msc_op_staggered(ctx, nc, dims, links, mass, flags)


# ----------------------------------------------------------------------------
# operator kernels
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("nc,dims", [(3, (4, 4, 4, 4)), (2, (6, 4, 2, 8)), (3, (8, 6, 4, 10))])
def test_staggered_apply_fp64_fp32(ctx, nc, dims):
    U = inputs.su_n_links(dims, nc, 0.7, 100 + nc)
    m, sig = 0.1, 0.3
    op = stag_op(ctx, U, dims, nc, m)
    assert msc.msc_op_recon(op) == 1
    n = inputs.volume(dims) * nc
    v = inputs.gaussian_source(n, 5)
    want = oracle.staggered_apply(U, dims, nc, m, v, sigma=sig)
    out = np.zeros_like(v)
    msc.msc_op_apply(ctx, op, sig, v, out, msc.MSC_FP64)
    assert rel(out, want) <= 1e-13
    out32 = np.zeros_like(v)
    msc.msc_op_apply(ctx, op, sig, v, out32, msc.MSC_FP32)
    assert rel(out32, want) <= 2e-6
    # D alone
    d = np.zeros_like(v)
    msc.msc_op_dslash(ctx, op, v, d)
    assert rel(d, oracle.dslash(U, dims, nc, v)) <= 1e-13
    msc.msc_op_destroy(op)


@pytest.mark.parametrize("nc", [2, 3])
def test_full_fp32_links_for_non_unitary(ctx, nc):
    dims = (4, 4, 4, 4)
    U = inputs.su_n_links(dims, nc, 0.7, 200 + nc)
    U = U * 1.01  # no longer unitary: reconstruction would be wrong
    op = stag_op(ctx, U, dims, nc, 0.2)
    assert msc.msc_op_recon(op) == 0
    n = inputs.volume(dims) * nc
    v = inputs.gaussian_source(n, 6)
    out32 = np.zeros_like(v)
    msc.msc_op_apply(ctx, op, 0.0, v, out32, msc.MSC_FP32)
    assert rel(out32, oracle.staggered_apply(U, dims, nc, 0.2, v)) <= 2e-6
    msc.msc_op_destroy(op)
    # the flag forces full storage for unitary links too
    op2 = stag_op(ctx, inputs.su_n_links(dims, nc, 0.7, 1), dims, nc, 0.2, msc.MSC_LINKS_FULL)
    assert msc.msc_op_recon(op2) == 0
    msc.msc_op_destroy(op2)


@pytest.mark.parametrize("nc,L", [(3, 4), (3, 6), (2, 6)])
def test_bsr_export_matches_stencil(ctx, nc, L):
    dims = (L, L, L, L)
    U = inputs.su_n_links(dims, nc, 0.8, 300 + L)
    m = 0.05
    op = stag_op(ctx, U, dims, nc, m)
    nbr, nnzb, bd = msc.msc_op_bsr_size(op)
    assert (nbr, nnzb, bd) == (inputs.volume(dims), 33 * inputs.volume(dims), nc)
    rp = np.zeros(nbr + 1, dtype=np.int64)
    ci = np.zeros(nnzb, dtype=np.int32)
    va = np.zeros((nnzb, bd, bd), dtype=np.complex128)
    msc.msc_staggered_export_bsr(ctx, op, rp, ci, va)
    n = nbr * bd
    v = inputs.gaussian_source(n, 7)
    # the exported matrix, applied by the oracle's plain BSR loop, is A
    assert rel(oracle.bsr_apply(rp, ci, va, v), oracle.staggered_apply(U, dims, nc, m, v)) <= 1e-13
    # and the GPU BSR kernels apply it in FP64 and FP32
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    want = oracle.staggered_apply(U, dims, nc, m, v, sigma=0.01)
    out = np.zeros_like(v)
    msc.msc_op_apply(ctx, bop, 0.01, v, out, msc.MSC_FP64)
    assert rel(out, want) <= 1e-13
    msc.msc_op_apply(ctx, bop, 0.01, v, out, msc.MSC_FP32)
    assert rel(out, want) <= 2e-6
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(op)


@pytest.mark.parametrize("bd,nbr", [(1, 37), (2, 70), (3, 33)])
def test_generic_bsr_apply_ragged(ctx, bd, nbr):
    rp, ci, va, A = inputs.random_hpd_bsr(nbr, bd, 5, 0.5, 400 + bd)
    n = nbr * bd
    v = inputs.gaussian_source(n, 8)
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    out = np.zeros_like(v)
    msc.msc_op_apply(ctx, bop, 0.2, v, out, msc.MSC_FP64)
    assert rel(out, A @ v + 0.2 * v) <= 1e-13
    # device-resident inputs give the same operator
    bop2 = msc.msc_op_bsr(ctx, nbr, bd, torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
                          torch.from_numpy(va).cuda())
    out2 = np.zeros_like(v)
    msc.msc_op_apply(ctx, bop2, 0.2, v, out2, msc.MSC_FP64)
    assert np.array_equal(out, out2)
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(bop2)


def test_bsr_rejects_bad_columns(ctx):
    rp, ci, va, A = inputs.random_hpd_bsr(10, 2, 3, 0.5, 9)
    bad = ci.copy()
    bad[3] = 10
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_bsr(ctx, 10, 2, rp, bad, va)
    assert e.value.code == msc.MSC_ERR_ARG


# ----------------------------------------------------------------------------
# solves
# ----------------------------------------------------------------------------

def check_solution(x, ref_x, rho, tol=1e-10, xtol=1e-8):
    for s in range(ref_x.shape[0]):
        assert rel(x[s], ref_x[s]) <= xtol, (s, rel(x[s], ref_x[s]))
    assert np.all(rho <= tol), rho


@pytest.mark.parametrize("prec", [msc.MSC_FP64, msc.MSC_MIXED])
def test_solve_4x4_su3_8shifts(ctx, prec):
    """The 4^4 SU(3) workload: every x_s against the oracle."""
    p = inputs.lattice_4x4_su3_8shifts()
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-13)
    ref_tol = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, p.tol)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    x, info = msc.solve(ctx, op, p.b[0], p.sigma, tol=p.tol, precision=prec)
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, x)
    check_solution(x, ref.x, rho)
    assert np.allclose(info.true_rel_resid[0], rho, rtol=1e-3, atol=1e-16)
    if prec == msc.MSC_FP64:
        # the same recurrences freeze the same shifts at the same iterations
        assert np.max(np.abs(info.shift_iters[0] - ref_tol.conv_iter)) <= 1
        assert abs(info.iters - ref_tol.iters) <= 1
    msc.msc_op_destroy(op)


def test_solve_multi_rhs_and_host_device_pointers(ctx):
    p = inputs.lattice_4x4_su3_8shifts(nrhs=3)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass, device=False)
    xh, _ = msc.solve(ctx, op, p.b, p.sigma, tol=p.tol, precision=msc.MSC_MIXED)
    bd = torch.from_numpy(p.b).cuda()
    xd, _ = msc.solve(ctx, op, bd, p.sigma, tol=p.tol, precision=msc.MSC_MIXED)
    assert np.array_equal(xh, xd.cpu().numpy())  # deterministic, pointer kind irrelevant
    for r in range(3):
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, 1e-13)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, xh[r])
        check_solution(xh[r], ref.x, rho)
    msc.msc_op_destroy(op)


@pytest.mark.parametrize("prec", [msc.MSC_FP64, msc.MSC_MIXED])
def test_solve_bsr_path_8x4(ctx, prec):
    """The 24^4 block-CSR recipe (m=0.05, eps=0.8, 15 shifts 1e-4..10) on an
    8^4 lattice: export, generic path, every x_s against the oracle."""
    p = inputs.lattice_24x4_su3_15shifts(L=8)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    nbr, nnzb, bd = msc.msc_op_bsr_size(op)
    rp = torch.zeros(nbr + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(nnzb, dtype=torch.int32, device="cuda")
    va = torch.zeros((nnzb, bd, bd), dtype=torch.complex128, device="cuda")
    msc.msc_staggered_export_bsr(ctx, op, rp, ci, va)
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-13)
    x, info = msc.solve(ctx, bop, p.b[0], p.sigma, tol=p.tol, precision=prec)
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, x)
    check_solution(x, ref.x, rho)
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(op)


@pytest.mark.parametrize("prec", [msc.MSC_FP64, msc.MSC_MIXED])
def test_solve_bsr_three_rhs(ctx, prec):
    """Several right-hand sides on the block-CSR path: the multi-shift stage
    applies the matrix to all of them in one launch (two systems per thread,
    an odd count leaves one group half empty); every x_s against the oracle."""
    p = inputs.lattice_24x4_su3_15shifts(L=6, nrhs=3)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    nbr, nnzb, bd = msc.msc_op_bsr_size(op)
    rp = torch.zeros(nbr + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(nnzb, dtype=torch.int32, device="cuda")
    va = torch.zeros((nnzb, bd, bd), dtype=torch.complex128, device="cuda")
    msc.msc_staggered_export_bsr(ctx, op, rp, ci, va)
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    x, info = msc.solve(ctx, bop, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol, precision=prec)
    assert info.status == 0
    x = x.cpu().numpy()
    for r in range(3):
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, 1e-13)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, x[r])
        check_solution(x[r], ref.x, rho)
    msc.msc_op_destroy(bop)
    msc.msc_op_destroy(op)


def test_generic_bsr_solve_ragged(ctx):
    rp, ci, va, A = inputs.random_hpd_bsr(45, 3, 6, 0.05, 77)
    n = A.shape[0]
    b = inputs.gaussian_source(n, 78)
    sig = inputs.log_shifts(1e-3, 3.0, 6)
    bop = msc.msc_op_bsr(ctx, 45, 3, rp, ci, va)
    for prec in (msc.MSC_FP64, msc.MSC_MIXED):
        x, info = msc.solve(ctx, bop, b, sig, tol=1e-10, precision=prec)
        for s, sv in enumerate(sig):
            xs = np.linalg.solve(A + sv * np.eye(n), b)
            assert rel(x[s], xs) <= 1e-8
            assert np.linalg.norm(b - (A @ x[s] + sv * x[s])) <= 1e-10 * np.linalg.norm(b)
    msc.msc_op_destroy(bop)


@pytest.mark.parametrize("bd,nbr", [(1, 613), (2, 301)])
def test_generic_bsr_one_rhs_small_blocks(ctx, bd, nbr):
    """One right-hand side on 1x1 and 2x2 complex blocks, mixed precision:
    the one-system FP32 SpMV (288-thread blocks, rows a grid's width apart)
    on block-row counts that fill neither a block nor a slice; every x_s
    against a dense FP64 solve."""
    rp, ci, va, A = inputs.random_hpd_bsr(nbr, bd, 7, 0.1, 500 + bd)
    n = A.shape[0]
    b = inputs.gaussian_source(n, 501 + bd)
    sig = inputs.log_shifts(1e-3, 3.0, 5)
    bop = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    x, info = msc.solve(ctx, bop, b, sig, tol=1e-10, precision=msc.MSC_MIXED)
    assert info.status == 0
    for s, sv in enumerate(sig):
        M = A + sv * np.eye(n)
        assert rel(x[s], np.linalg.solve(M, b)) <= 1e-8
        assert np.linalg.norm(b - M @ x[s]) <= 1e-10 * np.linalg.norm(b)
    msc.msc_op_destroy(bop)


@pytest.mark.parametrize("nrhs", [5, 19])
def test_generic_bsr_many_rhs_share_matrix(ctx, nrhs):
    """Right-hand sides sharing a ragged block-CSR matrix (45 block rows: one
    full slice and a ragged one) in mixed precision: each FP32 SpMV applies
    the matrix to every system still iterating, two per thread, one group of
    two per row of blocks (5 right-hand sides: three groups, the last half
    empty; 19: ten groups), and the refinement does the same for the shifts
    it refines. Every x_s against a dense FP64 solve."""
    rp, ci, va, A = inputs.random_hpd_bsr(45, 3, 6, 0.05, 91)
    n = A.shape[0]
    B = np.stack([inputs.gaussian_source(n, 100 + r) for r in range(nrhs)])
    sig = inputs.log_shifts(1e-3, 3.0, 4)
    bop = msc.msc_op_bsr(ctx, 45, 3, rp, ci, va)
    x, info = msc.solve(ctx, bop, B, sig, tol=1e-10, precision=msc.MSC_MIXED)
    assert info.status == 0
    for r in range(nrhs):
        for s, sv in enumerate(sig):
            M = A + sv * np.eye(n)
            assert rel(x[r][s], np.linalg.solve(M, B[r])) <= 1e-8
            assert np.linalg.norm(B[r] - M @ x[r][s]) <= 1e-10 * np.linalg.norm(B[r])
    msc.msc_op_destroy(bop)


def test_poisson_paper_operator_15_shifts(ctx):
    """The paper's own test operator (Sec. 4, Table 1): the 2-D five-point
    Poisson Laplacian, here on a 96 x 96 grid, 15 shifts 1e-4..10, through the
    generic block-CSR path with 1 x 1 blocks; every x_s against the oracle's
    CG-M (solved to 1e-13) and its FP64 true residual recomputed by the
    oracle. Also the single unshifted system (sigma = 0) of the comparison."""
    p = inputs.poisson_2d_15shifts(N=96)
    bop = msc.msc_op_bsr(ctx, p.n, 1, p.row_ptr, p.col_idx, p.vals)
    for sig in (p.sigma, np.array([0.0])):
        ref = oracle.cgm_bsr(p.row_ptr, p.col_idx, p.vals, p.b, sig, 1e-13)
        assert ref.status == 0
        for prec in (msc.MSC_FP64, msc.MSC_MIXED):
            x, info = msc.solve(ctx, bop, p.b, sig, tol=p.tol, precision=prec)
            assert info.status == 0
            for s, sv in enumerate(sig):
                r = p.b - oracle.bsr_apply(p.row_ptr, p.col_idx, p.vals, x[s], sigma=sv)
                assert np.linalg.norm(r) <= p.tol * np.linalg.norm(p.b), (prec, s)
                assert rel(x[s], ref.x[s]) <= 1e-8, (prec, s, rel(x[s], ref.x[s]))
    msc.msc_op_destroy(bop)


# ----------------------------------------------------------------------------
# edge cases
# ----------------------------------------------------------------------------

def test_zero_source_single_shift_and_zero_shift(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    b0 = np.zeros(p.n, dtype=np.complex128)
    x, info = msc.solve(ctx, op, b0, p.sigma)
    assert np.all(x == 0) and info.iters == 0 and info.status == 0
    # one shift, and a zero shift (A is positive definite for m > 0)
    for sig in ([0.0], [0.5], [0.0, 0.1]):
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], sig, 1e-13)
        x, info = msc.solve(ctx, op, p.b[0], sig)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], sig, x)
        check_solution(x, ref.x, rho)
    msc.msc_op_destroy(op)


def test_argument_and_breakdown_errors(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    with pytest.raises(msc.MscError) as e:
        msc.solve(ctx, op, p.b[0], [-0.1, 1.0])
    assert e.value.code == msc.MSC_ERR_ARG
    bad = p.b[0].copy()
    bad[5] = np.nan
    with pytest.raises(msc.MscError) as e:
        msc.solve(ctx, op, bad, p.sigma)
    assert e.value.code == msc.MSC_ERR_NONFINITE
    # iteration cap: status NOT_CONVERGED, x still written and finite
    x, info = msc.solve(ctx, op, p.b[0], p.sigma, max_iter=10, refine=0, raise_on_error=False)
    assert info.status == msc.MSC_ERR_NOT_CONVERGED and info.iters == 10
    assert np.all(np.isfinite(x)) and np.linalg.norm(x) > 0
    for prec in (msc.MSC_FP64, msc.MSC_MIXED):
        x, info = msc.solve(ctx, op, p.b[0], p.sigma, max_iter=0, precision=prec, raise_on_error=False)
        assert info.status == msc.MSC_ERR_NOT_CONVERGED and info.iters == 0 and np.all(x == 0)
    msc.msc_op_destroy(op)
    # an indefinite operator is reported as not positive definite
    rp, ci, va, A = inputs.random_hpd_bsr(12, 2, 3, 0.5, 5)
    neg = -va
    bop = msc.msc_op_bsr(ctx, 12, 2, rp, ci, neg)
    with pytest.raises(msc.MscError) as e:
        msc.solve(ctx, bop, inputs.gaussian_source(24, 3), [0.1])
    assert e.value.code == msc.MSC_ERR_NOT_HPD
    msc.msc_op_destroy(bop)


def test_maximum_shift_count_and_size_limits(ctx):
    """128 shifts (the most a system takes) in FP64 and mixed precision, each
    x_s against the oracle; 129 shifts, an empty operator and a block row
    longer than the kernels' 32-bit in-slice offsets allow are rejected."""
    p = inputs.lattice_4x4_su3_8shifts()
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    sig = inputs.log_shifts(1e-3, 10.0, 128)
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], sig, 1e-13)
    assert ref.status == 0
    for prec in (msc.MSC_FP64, msc.MSC_MIXED):
        x, info = msc.solve(ctx, op, p.b[0], sig, precision=prec)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], sig, x)
        check_solution(x, ref.x, rho)
    with pytest.raises(msc.MscError) as e:
        msc.solve(ctx, op, p.b[0], inputs.log_shifts(1e-3, 10.0, 129))
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(op)
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_bsr(ctx, 0, 1, np.zeros(1, np.int64), np.zeros(0, np.int32),
                       np.zeros((0, 1, 1), np.complex128))
    assert e.value.code == msc.MSC_ERR_ARG
    # one block row of 2^26 / 9 + 1 blocks of 3 x 3: beyond the limit
    m = (1 << 26) // 9 + 1
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_bsr(ctx, 1, 3, np.array([0, m], np.int64), np.zeros(m, np.int32),
                       np.zeros((m, 3, 3), np.complex128))
    assert e.value.code == msc.MSC_ERR_ARG


def test_no_freeze_matches_freeze(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    x1, i1 = msc.solve(ctx, op, p.b[0], p.sigma, precision=msc.MSC_FP64, freeze=True)
    x2, i2 = msc.solve(ctx, op, p.b[0], p.sigma, precision=msc.MSC_FP64, freeze=False)
    for s in range(len(p.sigma)):
        assert rel(x1[s], x2[s]) <= 1e-8
    msc.msc_op_destroy(op)


def test_context_reuse_across_sizes(ctx):
    """Solves of different sizes on one context (workspace layout changes
    between them) give the same answers as on a fresh context."""
    rp, ci, va, A = inputs.random_hpd_bsr(45, 3, 6, 0.05, 77)
    b = inputs.gaussian_source(135, 78)
    sig = inputs.log_shifts(1e-3, 3.0, 6)
    p = inputs.lattice_24x4_su3_15shifts(L=4)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    bop = msc.msc_op_bsr(ctx, 45, 3, rp, ci, va)
    for prec in (msc.MSC_FP64, msc.MSC_MIXED):
        msc.solve(ctx, op, p.b[0], p.sigma, precision=prec)
        x, info = msc.solve(ctx, bop, b, sig, precision=prec)
        assert info.status == 0
        for s, sv in enumerate(sig):
            assert np.linalg.norm(b - (A @ x[s] + sv * x[s])) <= 1e-10 * np.linalg.norm(b)
        x2, _ = msc.solve(ctx, op, p.b[0], p.sigma, precision=prec)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, x2)
        assert np.all(rho <= 1e-10)
    msc.msc_op_destroy(op)
    msc.msc_op_destroy(bop)


def test_mixed_reliable_updates_keep_fast_convergence_stable(ctx):
    """A small SU(2) lattice whose residual falls by several decades between
    fixed-period reliable updates: with updates triggered by the residual's
    fall (delta 0.01) the mixed solve converges for every right-hand side."""
    p = inputs.staggered_problem((6, 4, 4, 6), 2, 0.05, 0.6, inputs.log_shifts(1e-4, 1.0, 8), 2,
                                 1e-10, 7010)
    op = stag_op(ctx, p.links, p.dims, p.nc, p.mass)
    for r in range(2):
        x, info = msc.solve(ctx, op, p.b[r], p.sigma, precision=msc.MSC_MIXED)
        assert info.status == 0 and info.reliable_updates > 0
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, 1e-13)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, x)
        check_solution(x, ref.x, rho)
    msc.msc_op_destroy(op)
