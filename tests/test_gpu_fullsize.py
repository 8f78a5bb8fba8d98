"""Parity at the benchmark's full size and launch configuration: the 24^4
SU(3) staggered operator exported as block-CSR (331,776 block rows), 15
shifts 1e-4..10, mixed precision, tolerance 1e-10 — exactly what bench.py
times. Every x_s is compared with the FP64 oracle's CG-M solution (solved to
its floor) and every shift's FP64 true residual is recomputed by the oracle
from the returned x_s."""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402


@pytest.fixture(scope="module")
def problem():
    return inputs.lattice_24x4_su3_15shifts()


def test_fullsize_bsr_mixed_against_oracle(problem):
    p = problem
    ctx = msc.msc_create(0, torch.cuda.current_stream())
    sop = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    nbr, nnzb, bd = msc.msc_op_bsr_size(sop)
    rp = torch.empty(nbr + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(nnzb, dtype=torch.int32, device="cuda")
    va = torch.empty((nnzb, bd, bd), dtype=torch.complex128, device="cuda")
    msc.msc_staggered_export_bsr(ctx, sop, rp, ci, va)
    op = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    del va, rp, ci
    x, info = msc.solve(ctx, op, torch.from_numpy(p.b[0]).cuda(), p.sigma, tol=p.tol,
                        precision=msc.MSC_MIXED)
    x = x.cpu().numpy()
    assert info.status == 0
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, x)
    assert np.all(rho <= p.tol), rho
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-13)
    for s in range(len(p.sigma)):
        err = np.linalg.norm(x[s] - ref.x[s]) / np.linalg.norm(ref.x[s])
        assert err <= 1e-8, (s, err)
    msc.msc_op_destroy(op)
    msc.msc_op_destroy(sop)
    msc.msc_destroy(ctx)
