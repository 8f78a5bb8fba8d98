"""Parity of the staggered stencil path on the large production-shaped
workload: 32^4 SU(3) (1,048,576 sites, 3,145,728 complex unknowns), m = 0.01,
eps = 0.9, 20 shifts log-spaced 1e-5..10, 8 Gaussian right-hand sides, mixed
precision (FP32 stencil passes and vector updates, FP64 recurrences, dot
products and reliable updates every 50 iterations at the latest), tolerance
1e-10 on the FP64 true residual of every shift.

At full size the oracle cannot solve the 160 systems in test time, so it
checks what it can compute one by one: the FP64 true residual
|b - (A + sigma_s) x_s| / |b| of sampled solutions, recomputed on the CPU
from the returned x_s. The same recipe on an 8^4 lattice is compared with the
oracle's own CG-M solution element by element. A solve in a second context
(on memory the first one freed, filled with NaN patterns in between) must
reproduce the first bit for bit.

Error bound used for x_s: A = m^2 + D^dag D with |D| <= 4 for unitary links,
so the spectrum of A + sigma lies in [m^2 + sigma, m^2 + 16 + sigma] and
|x_s - x_s*| / |x_s*| <= kappa_s (rho_s + rho_s*), kappa_s the ratio of the
ends, rho the two solutions' true relative residuals.
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402


def kappa(mass, sigma):
    return (mass ** 2 + 16.0 + sigma) / (mass ** 2 + sigma)


@pytest.fixture(scope="module")
def ctx():
    msc.load()
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


def test_32x4_8rhs_20shifts_mixed_true_residuals(ctx):
    p = inputs.lattice_32x4_su3_20shifts()
    R, S, n = p.b.shape[0], len(p.sigma), p.n
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    assert msc.msc_op_recon(op) == 1
    b = torch.from_numpy(p.b).cuda()
    x, info = msc.solve(ctx, op, b, p.sigma, tol=p.tol, precision=msc.MSC_MIXED)
    assert info.status == 0
    assert info.true_rel_resid.shape == (R, S)
    assert np.all(info.true_rel_resid <= p.tol), info.true_rel_resid.max()
    assert info.reliable_updates > 0
    # every right-hand side: its hardest and its easiest shift, plus one drawn
    g = inputs.rng(4003)
    for r in range(R):
        for s in sorted({0, S - 1, int(g.integers(1, S - 1))}):
            xs = x[r, s].cpu().numpy()
            rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r],
                                                 p.sigma[s:s + 1], xs[None, :])[0]
            assert rho <= p.tol, (r, s, rho)
            # the library's own FP64 residual of that solution agrees
            assert abs(rho - info.true_rel_resid[r, s]) <= 1e-3 * p.tol, (r, s, rho)
    msc.msc_op_destroy(op)


def test_32x4_recipe_on_8x4_matches_oracle_solution(ctx):
    p = inputs.lattice_32x4_su3_20shifts(L=8)
    R, S = p.b.shape[0], len(p.sigma)
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    x, info = msc.solve(ctx, op, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol,
                        precision=msc.MSC_MIXED)
    assert info.status == 0
    x = x.cpu().numpy()
    worst = 0.0
    for r in range(R):
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, 1e-13)
        assert ref.status == 0
        rho_ref = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, ref.x)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, x[r])
        assert np.all(rho <= p.tol), rho
        for s in range(S):
            err = np.linalg.norm(x[r, s] - ref.x[s]) / np.linalg.norm(ref.x[s])
            bound = kappa(p.mass, p.sigma[s]) * (rho[s] + rho_ref[s])
            assert err <= bound, (r, s, err, bound)
            assert err <= 1e-8, (r, s, err, bound)
            worst = max(worst, err)
    msc.msc_op_destroy(op)
    print(f"worst x_s error {worst:.2e}")


def test_second_context_on_recycled_memory_repeats_the_solve():
    """Workspace zeroing must be ordered before the solve's kernels: a new
    context whose buffers reuse freed (here NaN-filled) device memory gives
    the same solution as the first context, bit for bit."""
    p = inputs.lattice_32x4_su3_20shifts(L=24, nrhs=8)
    outs = []
    for trial in range(2):
        c = msc.msc_create(0, torch.cuda.current_stream())
        op = msc.msc_op_staggered(c, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
        x, info = msc.solve(c, op, torch.from_numpy(p.b).cuda(), p.sigma, tol=p.tol,
                            precision=msc.MSC_MIXED)
        assert info.status == 0 and np.all(info.true_rel_resid <= p.tol)
        outs.append((x.cpu().numpy(), info.iters, info.refine_iters))
        msc.msc_op_destroy(op)
        msc.msc_destroy(c)
        del x
        # fill what the context freed with NaN bit patterns
        junk = torch.full((3 << 28,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        del junk
        torch.cuda.empty_cache()
    (x0, i0, r0), (x1, i1, r1) = outs
    assert (i0, r0) == (i1, r1)
    assert np.array_equal(x0, x1)
