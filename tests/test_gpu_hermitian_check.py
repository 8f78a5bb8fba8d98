"""MSC_CHECK_HERMITIAN: msc_op_bsr's on-device check that A = A^dagger
(CG-M, Sec. 2, solves the shifted family of eq. linprob for Hermitian A).

Accepted: random Hermitian positive-definite block-CSR matrices (ragged
patterns, bd = 1, 2, 3), the staggered operator's own export (blocks of (i, j)
and (j, i) assembled along different paths, equal to rounding), and a matrix
that stores one entry as two repeated blocks that only sum to the Hermitian
value. Refused with MSC_ERR_NOT_HPD: one entry perturbed by 1e-9 relative,
a block whose transposed partner is missing, and a non-Hermitian matrix,
which msc_solve_nonherm still takes without the flag.
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


def _create(ctx, nbr, bd, rp, ci, va, flags=msc.MSC_CHECK_HERMITIAN):
    return msc.msc_op_bsr(ctx, nbr, bd, rp, ci, np.ascontiguousarray(va), flags)


def _refused(ctx, nbr, bd, rp, ci, va):
    with pytest.raises(msc.MscError) as e:
        _create(ctx, nbr, bd, rp, ci, va)
    assert e.value.code == msc.MSC_ERR_NOT_HPD


@pytest.mark.parametrize("bd", [1, 2, 3])
def test_hermitian_matrices_pass_and_solve(ctx, bd):
    nbr = 37
    rp, ci, va, A = inputs.random_hpd_bsr(nbr, bd, 5, 0.5, 40 + bd)
    op = _create(ctx, nbr, bd, rp, ci, va)
    b = inputs.gaussian_source(nbr * bd, 50 + bd)
    sig = np.array([0.0, 0.3])
    x, info = msc.solve(ctx, op, b, sig, tol=1e-10, precision=msc.MSC_FP64)
    assert info.status == 0
    for s, sg in enumerate(sig):
        ref = np.linalg.solve(A + sg * np.eye(A.shape[0]), b)
        assert np.linalg.norm(x[s] - ref) <= 1e-8 * np.linalg.norm(ref)
    msc.msc_op_destroy(op)


def test_staggered_export_passes(ctx):
    p = inputs.lattice_4x4_su3_8shifts()
    sop = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    nbr, nnzb, bd = msc.msc_op_bsr_size(sop)
    rp = np.empty(nbr + 1, dtype=np.int64)
    ci = np.empty(nnzb, dtype=np.int32)
    va = np.empty((nnzb, bd, bd), dtype=np.complex128)
    msc.msc_staggered_export_bsr(ctx, sop, rp, ci, va)
    op = _create(ctx, nbr, bd, rp, ci, va)
    msc.msc_op_destroy(op)
    msc.msc_op_destroy(sop)


def test_repeated_columns_are_summed_before_the_check(ctx):
    rp, ci, va, _ = inputs.random_hpd_bsr(12, 2, 3, 1.0, 60)
    # split every diagonal block into two stored blocks: a + (d - a), where a
    # alone is not Hermitian
    g = inputs.rng(61)
    rows, cols, vals = [0], [], []
    for i in range(12):
        for k in range(rp[i], rp[i + 1]):
            if ci[k] == i:
                a = g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))
                cols += [i, i]
                vals += [a, va[k] - a]
            else:
                cols.append(ci[k])
                vals.append(va[k])
        rows.append(len(cols))
    rp2 = np.asarray(rows, dtype=np.int64)
    ci2 = np.asarray(cols, dtype=np.int32)
    va2 = np.asarray(vals, dtype=np.complex128)
    op = _create(ctx, 12, 2, rp2, ci2, va2)
    msc.msc_op_destroy(op)
    # the same split with one half perturbed is refused
    va2[1, 0, 1] += 1e-3
    _refused(ctx, 12, 2, rp2, ci2, va2)


def test_perturbed_entry_is_refused(ctx):
    rp, ci, va, _ = inputs.random_hpd_bsr(40, 3, 4, 0.5, 70)
    # an off-diagonal entry of an off-diagonal block, off by 1e-9 relative
    k = next(k for k in range(len(ci)) if ci[k] != 0 and k >= rp[1])
    va = va.copy()
    va[k, 0, 2] += 1e-9 * np.abs(va).max()
    _refused(ctx, 40, 3, rp, ci, va)


def test_missing_partner_is_refused(ctx):
    # tridiagonal Hermitian pattern with one (i, i+1) block removed
    nbr, bd = 10, 1
    rows, cols, vals = [0], [], []
    for i in range(nbr):
        for j in (i - 1, i, i + 1):
            if 0 <= j < nbr and not (i == 3 and j == 4):
                cols.append(j)
                vals.append(np.array([[4.0 if i == j else -1.0]], dtype=np.complex128))
        rows.append(len(cols))
    rp = np.asarray(rows, dtype=np.int64)
    ci = np.asarray(cols, dtype=np.int32)
    va = np.asarray(vals, dtype=np.complex128)
    _refused(ctx, nbr, bd, rp, ci, va)


def test_nonhermitian_matrix_refused_with_flag_solved_without(ctx):
    rp, ci, va, A = inputs.random_nonhermitian_bsr(30, 2, 4, 0.5, 0.3, 80)
    _refused(ctx, 30, 2, rp, ci, va)
    op = msc.msc_op_bsr(ctx, 30, 2, rp, ci, va)
    b = inputs.gaussian_source(60, 81)
    sig = np.array([0.0, 0.2, 1.0])
    x, info = msc.solve_nonherm(ctx, op, torch.from_numpy(b).cuda(), sig, tol=1e-10)
    assert info.status == 0
    ref = oracle.bicgstabm_bsr(rp, ci, va, b, sig, 1e-13)
    xs = x.cpu().numpy()
    for s in range(len(sig)):
        assert np.linalg.norm(xs[s] - ref.x[s]) <= 1e-8 * np.linalg.norm(ref.x[s])
    msc.msc_op_destroy(op)


def test_unknown_flag_bits_are_refused(ctx):
    rp, ci, va, _ = inputs.random_hpd_bsr(8, 1, 2, 1.0, 90)
    with pytest.raises(msc.MscError) as e:
        msc.msc_op_bsr(ctx, 8, 1, rp, ci, va, 4)
    assert e.value.code == msc.MSC_ERR_ARG
