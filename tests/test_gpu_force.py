"""Adjoint of S = sum_s c_s Re(phi^dag (A + sigma_s)^{-1} phi) on the GPU.

The 16^4 SU(3) force workload: m = 0.05, eps = 0.7, 12 shifts log-spaced
1e-4..5 with c_s = sigma_s^0.5 / 12, Gaussian phi.
  * the force kernel against the oracle's force on the same vectors (FP64,
    rounding-order tolerance 1e-12 relative);
  * the autograd gradients (mixed-precision solve) against the FP64 CPU
    gradient from the oracle's own solve, and against central differences
    with step 1e-6 on 32 random link entries (real and imaginary parts),
    to 1e-6 relative. The differences are written without cancellation:
    S(U+) - S(U-) = sum_s c_s x_s(U+)^dag (A(U-) - A(U+)) x_s(U-).
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1102_2143_gb300 as msc  # noqa: E402
from paper_1102_2143_gb300.autograd import quad_form  # noqa: E402


@pytest.fixture(scope="module")
def work():
    p, c = inputs.lattice_16x4_su3_force()
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-12)
    assert ref.status == 0
    return p, c, ref


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_force_kernel_matches_oracle_on_same_vectors(work):
    p, c, ref = work
    h = msc.default_context(0)
    op = msc.msc_op_staggered(h, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    S = len(p.sigma)
    xs = inputs.gaussian_source(p.n, 77, nrhs=S)  # any vectors: the force is algebraic in x
    dU = np.zeros_like(p.links)
    dphi = np.zeros(p.n, dtype=np.complex128)
    msc.msc_quad_form_grad(h, op, S, c, xs, dphi, dU)
    assert rel(dU, oracle.link_force(p.links, p.dims, p.nc, c, xs)) <= 1e-12
    assert rel(dphi, 2 * np.tensordot(c, xs, axes=1)) <= 1e-13
    val = msc.msc_quad_form(h, op, p.b[0], S, c, ref.x)
    assert abs(val - oracle.quad_form(p.b[0], ref.x, c)) <= 1e-12 * abs(val)
    msc.msc_op_destroy(op)


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_matches_fp64_cpu_gradient(work, recompute):
    p, c, ref = work
    phi = torch.from_numpy(p.b[0]).cuda().requires_grad_(True)
    U = torch.from_numpy(p.links).cuda().requires_grad_(True)
    Sv = quad_form(phi, U, p.sigma, c, p.dims, p.nc, p.mass, tol=1e-10,
                   precision=msc.MSC_MIXED, recompute=recompute)
    Sv.backward()
    want_S = oracle.quad_form(p.b[0], ref.x, c)
    assert abs(Sv.item() - want_S) <= 1e-9 * abs(want_S)
    G = oracle.link_force(p.links, p.dims, p.nc, c, ref.x)
    assert rel(U.grad.cpu().numpy(), G) <= 1e-6
    assert rel(phi.grad.cpu().numpy(), 2 * np.tensordot(c, ref.x, axes=1)) <= 1e-6


def test_link_gradient_matches_central_differences(work):
    p, c, ref = work
    h = msc.default_context(0)
    phi = torch.from_numpy(p.b[0]).cuda()
    U = torch.from_numpy(p.links).cuda().requires_grad_(True)
    quad_form(phi, U, p.sigma, c, p.dims, p.nc, p.mass, tol=1e-10).backward()
    grad = U.grad.cpu().numpy()
    g = inputs.rng(3003)
    V = inputs.volume(p.dims)
    step = 1e-6
    worst = 0.0
    for _ in range(32):
        mu, site = int(g.integers(4)), int(g.integers(V))
        a, b = int(g.integers(p.nc)), int(g.integers(p.nc))
        for d in (1.0, 1j):
            Up, Um = p.links.copy(), p.links.copy()
            Up[mu, site, a, b] += d * step
            Um[mu, site, a, b] -= d * step
            opp = msc.msc_op_staggered(h, p.nc, p.dims, Up, p.mass)
            opm = msc.msc_op_staggered(h, p.nc, p.dims, Um, p.mass)
            xp, _ = msc.solve(h, opp, p.b[0], p.sigma, tol=1e-12, precision=msc.MSC_FP64)
            xm, _ = msc.solve(h, opm, p.b[0], p.sigma, tol=1e-12, precision=msc.MSC_FP64)
            tot = 0.0
            for s in range(len(p.sigma)):
                am = np.zeros(p.n, dtype=np.complex128)
                ap = np.zeros(p.n, dtype=np.complex128)
                msc.msc_op_apply(h, opm, 0.0, xm[s], am, msc.MSC_FP64)
                msc.msc_op_apply(h, opp, 0.0, xm[s], ap, msc.MSC_FP64)
                tot += c[s] * np.vdot(xp[s], am - ap).real
            fd = tot / (2 * step)
            got = grad[mu, site, a, b].real if d == 1.0 else grad[mu, site, a, b].imag
            scale = max(abs(got), 1e-3 * np.abs(grad).max())
            worst = max(worst, abs(got - fd) / scale)
            msc.msc_op_destroy(opp)
            msc.msc_op_destroy(opm)
    assert worst <= 1e-6, worst
