"""Pins of the FP64 oracle against facts fixed by the mathematics.

Each test checks the oracle against something other than itself: a closed
form, a dense LAPACK solve, textbook CG, an exact identity of the operator,
or brute force on a tiny case. Together they are chosen so that a dropped
term, a wrong sign, a wrong index or a transposed link fails at least one.
"""
import numpy as np
import pytest

import oracle
from paper_1102_2143_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def _vec(n, seed):
    return inputs.gaussian_source(n, seed)


# ----------------------------------------------------------------------------
# Operator structure (staggered D, A = m^2 - D^2)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_dslash_is_anti_hermitian(nc):
    dims = (4, 4, 6, 4)
    U = inputs.su_n_links(dims, nc, 0.7, 11)
    n = inputs.volume(dims) * nc
    u, v = _vec(n, 1), _vec(n, 2)
    Du = oracle.dslash(U, dims, nc, u)
    Dv = oracle.dslash(U, dims, nc, v)
    lhs = np.vdot(u, Dv)
    rhs = -np.vdot(Du, v)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # <v, D v> purely imaginary
    q = np.vdot(v, Dv)
    assert abs(q.real) <= 1e-13 * np.linalg.norm(v) ** 2


def test_a_hermitian_positive():
    dims, nc, m = (4, 4, 4, 4), 3, 0.1
    U = inputs.su_n_links(dims, nc, 0.9, 12)
    n = inputs.volume(dims) * nc
    u, v = _vec(n, 3), _vec(n, 4)
    Au = oracle.staggered_apply(U, dims, nc, m, u)
    Av = oracle.staggered_apply(U, dims, nc, m, v)
    assert abs(np.vdot(u, Av) - np.vdot(Au, v)) <= 1e-13 * abs(np.vdot(u, Av))
    Dv = oracle.dslash(U, dims, nc, v)
    vAv = np.vdot(v, Av)
    assert abs(vAv.imag) <= 1e-13 * abs(vAv)
    # <v, A v> = m^2 |v|^2 + |D v|^2  >=  m^2 |v|^2
    expect = m * m * np.linalg.norm(v) ** 2 + np.linalg.norm(Dv) ** 2
    assert abs(vAv.real - expect) <= 1e-12 * expect
    assert vAv.real >= m * m * np.linalg.norm(v) ** 2


def _unit(n, i):
    e = np.zeros(n, dtype=np.complex128)
    e[i] = 1.0
    return e


def _site(x, dims):
    return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))


@pytest.mark.parametrize("nc", [2, 3])
def test_a_blocks_diagonal_and_two_hop(nc):
    """A_xx = (m^2 + 2) I for unitary links; the block coupling x to x+2mu is
    -1/4 U_mu(x) U_mu(x+mu) (the single two-hop path); that to x+mu+nu is the
    sum of the two paths with the staggered phases."""
    dims, m = (6, 6, 6, 6), 0.3
    U = inputs.su_n_links(dims, nc, 0.8, 13)
    n = inputs.volume(dims) * nc
    x = (1, 2, 3, 4)
    sx = _site(x, dims)
    for mu in range(4):
        xp = list(x); xp[mu] = (xp[mu] + 1) % dims[mu]
        x2 = list(x); x2[mu] = (x2[mu] + 2) % dims[mu]
        s1, s2 = _site(xp, dims), _site(x2, dims)
        blk = np.zeros((nc, nc), dtype=np.complex128)
        for b in range(nc):
            col = oracle.staggered_apply(U, dims, nc, m, _unit(n, s2 * nc + b))
            blk[:, b] = col[sx * nc:(sx + 1) * nc]
        expect = -0.25 * U[mu, sx] @ U[mu, s1]
        assert np.max(np.abs(blk - expect)) <= 1e-14
    diag = np.zeros((nc, nc), dtype=np.complex128)
    for b in range(nc):
        col = oracle.staggered_apply(U, dims, nc, m, _unit(n, sx * nc + b))
        diag[:, b] = col[sx * nc:(sx + 1) * nc]
    assert np.max(np.abs(diag - (m * m + 2.0) * np.eye(nc))) <= 1e-14
    # x -> x + e0 + e1: paths via x+e0 and via x+e1.
    # eta_0 = 1; eta_1(x) = (-1)^x0.
    def eta(y, mu):
        return (-1) ** (sum(y[:mu]) % 2)
    y0 = list(x); y0[0] += 1
    y1 = list(x); y1[1] += 1
    z = list(x); z[0] += 1; z[1] += 1
    sz, sy0, sy1 = _site(z, dims), _site(y0, dims), _site(y1, dims)
    blk = np.zeros((nc, nc), dtype=np.complex128)
    for b in range(nc):
        col = oracle.staggered_apply(U, dims, nc, m, _unit(n, sz * nc + b))
        blk[:, b] = col[sx * nc:(sx + 1) * nc]
    expect = -0.25 * (eta(x, 0) * eta(y0, 1) * U[0, sx] @ U[1, sy0]
                      + eta(x, 1) * eta(y1, 0) * U[1, sx] @ U[0, sy1])
    assert np.max(np.abs(blk - expect)) <= 1e-14


def _free_field_solution(b, dims, nc, m, sigma):
    """(m^2 + sigma - D^2)^{-1} b for U = 1 in momentum space: the staggered
    phases make the cross terms of D^2 cancel, leaving
    -D^2 = sum_mu sin^2(p_mu), p_mu = 2 pi k / L_mu."""
    L0, L1, L2, L3 = dims
    bb = b.reshape(L3, L2, L1, L0, nc)
    bh = np.fft.fftn(bb, axes=(0, 1, 2, 3))
    k = [2 * np.pi * np.fft.fftfreq(L) for L in (L3, L2, L1, L0)]
    P = np.meshgrid(*k, indexing="ij")
    lam = m * m + sigma + sum(np.sin(p) ** 2 for p in P)
    xh = bh / lam[..., None]
    return np.fft.ifftn(xh, axes=(0, 1, 2, 3)).reshape(-1)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 8)])
def test_free_field_closed_form(dims):
    nc, m = 3, 0.2
    U = inputs.su_n_links(dims, nc, 0.0, 14)
    assert np.all(U == np.eye(nc))
    n = inputs.volume(dims) * nc
    b = _vec(n, 5)
    sig = inputs.log_shifts(1e-2, 1.0, 4)
    for s in sig:
        xs = _free_field_solution(b, dims, nc, m, s)
        # the oracle's operator maps the closed-form solution back to b
        back = oracle.staggered_apply(U, dims, nc, m, xs, sigma=s)
        assert np.linalg.norm(back - b) <= 1e-13 * np.linalg.norm(b)
    res = oracle.cgm_staggered(U, dims, nc, m, b, sig, 1e-13)
    assert res.status == 0
    for i, s in enumerate(sig):
        xs = _free_field_solution(b, dims, nc, m, s)
        assert np.linalg.norm(res.x[i] - xs) <= 1e-11 * np.linalg.norm(xs)


def test_gauge_covariance():
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dagger gives A' = G A G^dagger."""
    dims, nc, m = (4, 4, 4, 6), 3, 0.15
    U = inputs.su_n_links(dims, nc, 0.6, 15)
    g = inputs.random_gauge(dims, nc, 16)
    V = inputs.volume(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        sites = np.arange(V)
        coords = np.stack(np.unravel_index(sites, (dims[3], dims[2], dims[1], dims[0]))[::-1], 1)
        c2 = coords.copy()
        c2[:, mu] = (c2[:, mu] + 1) % dims[mu]
        fwd = c2[:, 0] + dims[0] * (c2[:, 1] + dims[1] * (c2[:, 2] + dims[2] * c2[:, 3]))
        Up[mu] = g @ U[mu] @ np.conj(np.swapaxes(g[fwd], 1, 2))
    n = V * nc
    v = _vec(n, 6)
    Gv = (g @ v.reshape(V, nc, 1)).reshape(-1)
    lhs = oracle.staggered_apply(Up, dims, nc, m, Gv)
    rhs = (g @ oracle.staggered_apply(U, dims, nc, m, v).reshape(V, nc, 1)).reshape(-1)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)
    # a transposed link breaks covariance: the pin is sensitive to it
    UT = np.swapaxes(U, 2, 3).copy()
    UpT = np.swapaxes(Up, 2, 3).copy()
    bad = oracle.staggered_apply(UpT, dims, nc, m, Gv)
    badr = (g @ oracle.staggered_apply(UT, dims, nc, m, v).reshape(V, nc, 1)).reshape(-1)
    assert np.linalg.norm(bad - badr) > 1e-3 * np.linalg.norm(badr)


# ----------------------------------------------------------------------------
# CG-M recurrences
# ----------------------------------------------------------------------------

def _dense_A(U, dims, nc, m):
    n = inputs.volume(dims) * nc
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        A[:, j] = oracle.staggered_apply(U, dims, nc, m, _unit(n, j))
    return A


def test_cgm_matches_dense_solve_4x4_su3():
    """The 4^4 SU(3) workload (768 unknowns, 8 shifts): CG-M equals LAPACK."""
    p = inputs.lattice_4x4_su3_8shifts()
    A = _dense_A(p.links, p.dims, p.nc, p.mass)
    assert np.max(np.abs(A - np.conj(A.T))) < 1e-15
    assert np.linalg.eigvalsh(A).min() > 0.9 * p.mass ** 2
    b = p.b[0]
    res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, 1e-13)
    assert res.status == 0
    n = A.shape[0]
    for i, s in enumerate(p.sigma):
        xs = np.linalg.solve(A + s * np.eye(n), b)
        assert np.linalg.norm(res.x[i] - xs) <= 1e-11 * np.linalg.norm(xs)
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, res.x)
    assert np.all(rho <= 1e-12)


def test_cgm_iterates_equal_textbook_cg():
    """x_s after k CG-M iterations equals k iterations of textbook CG on
    A + sigma_s (same Krylov space, same Galerkin condition)."""
    p = inputs.lattice_4x4_su3_8shifts()
    b = p.b[0]
    for k in (1, 2, 3, 7, 15, 25):
        res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, 0.0, max_iter=k,
                                   freeze=False)
        assert res.iters == k
        for i, s in enumerate(p.sigma):
            xc, it, st = oracle.cg_staggered(p.links, p.dims, p.nc, p.mass, b, s, 0.0, max_iter=k)
            assert it == k
            assert np.linalg.norm(res.x[i] - xc) <= 1e-11 * np.linalg.norm(xc)


def test_cgm_first_iteration_hand_check():
    """After one iteration x_s = R/(P + sigma R) b, the exact shifted CG step."""
    p = inputs.lattice_4x4_su3_8shifts()
    b = p.b[0]
    res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, 0.0, max_iter=1,
                               freeze=False)
    R = np.vdot(b, b).real
    P = np.vdot(b, oracle.staggered_apply(p.links, p.dims, p.nc, p.mass, b)).real
    for i, s in enumerate(p.sigma):
        assert np.linalg.norm(res.x[i] - R / (P + s * R) * b) <= 1e-14 * np.linalg.norm(res.x[i])
        assert abs(res.zeta[i] - 1.0 / (1.0 + s * R / P)) <= 1e-15


def test_cgm_collinear_residuals():
    """b - (A + sigma_s) x_s = zeta_s r at every iteration."""
    p = inputs.lattice_4x4_su3_8shifts()
    b = p.b[0]
    for k in (4, 12, 30):
        res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, 0.0, max_iter=k,
                                   freeze=False)
        for i, s in enumerate(p.sigma):
            rs = b - oracle.staggered_apply(p.links, p.dims, p.nc, p.mass, res.x[i], sigma=s)
            assert np.linalg.norm(rs - res.zeta[i] * res.r) <= 1e-11 * np.linalg.norm(b)


def test_cgm_freeze_reports_per_shift_iterations():
    p = inputs.lattice_4x4_su3_8shifts()
    b = p.b[0]
    res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, p.tol)
    assert res.status == 0
    # larger shifts are better conditioned and converge no later
    assert np.all(np.diff(res.conv_iter) <= 0)
    assert res.iters == res.conv_iter.max()
    rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, res.x)
    assert np.all(rho <= 5 * p.tol)
    # freezing changes nothing but the work: compare with the paper's behaviour
    res2 = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, p.tol, freeze=False)
    for i in range(len(p.sigma)):
        assert np.linalg.norm(res.x[i] - res2.x[i]) <= 1e-9 * np.linalg.norm(res2.x[i])


def test_true_residual_exact_values():
    """rho_s = |b - (A + sigma_s) x_s| / |b| on solutions with a planted
    residual: x_s = (A + sigma_s)^{-1} (b - e_s) by LAPACK gives rho_s =
    |e_s| / |b| exactly (to rounding). The planted norms differ by orders of
    magnitude per shift, so a wrong shift index, a wrong normalisation (|b|^2,
    no square root) or a dropped sigma fails; x = 0 gives rho = 1."""
    dims, nc, m = (2, 2, 4, 2), 2, 0.3
    U = inputs.su_n_links(dims, nc, 0.8, 14)
    A = _dense_A(U, dims, nc, m)
    n = A.shape[0]
    b = _vec(n, 15)
    sigma = np.array([0.0, 0.05, 2.0])
    scale = np.array([1e-2, 1e-4, 1e-6])
    x = np.empty((len(sigma), n), dtype=np.complex128)
    want = np.empty(len(sigma))
    for i, s in enumerate(sigma):
        e = _vec(n, 16 + i)
        e *= scale[i] * np.linalg.norm(b) / np.linalg.norm(e)
        x[i] = np.linalg.solve(A + s * np.eye(n), b - e)
        want[i] = np.linalg.norm(e) / np.linalg.norm(b)
    rho = oracle.true_residual_staggered(U, dims, nc, m, b, sigma, x)
    assert np.allclose(rho, want, rtol=1e-6, atol=0), (rho, want)
    # the pairing of x_s with sigma_s matters
    rho_swapped = oracle.true_residual_staggered(U, dims, nc, m, b, sigma, x[::-1].copy())
    assert not np.allclose(rho_swapped, want[::-1], rtol=1e-2, atol=0)
    rho0 = oracle.true_residual_staggered(U, dims, nc, m, b, sigma, np.zeros_like(x))
    assert np.allclose(rho0, 1.0, rtol=1e-15, atol=0)


def test_quadratic_form_bounds():
    """|phi|^2/(m^2+16+sigma) <= phi^dagger (A+sigma)^-1 phi <= |phi|^2/(m^2+sigma)
    since 0 <= -D^2 <= 16 for unitary links (|D| <= 4)."""
    p = inputs.lattice_4x4_su3_8shifts()
    b = p.b[0]
    res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, 1e-12)
    nb2 = np.vdot(b, b).real
    for i, s in enumerate(p.sigma):
        q = np.vdot(b, res.x[i]).real
        assert nb2 / (p.mass ** 2 + 16 + s) <= q <= nb2 / (p.mass ** 2 + s)


def test_zero_source_gives_zero():
    p = inputs.lattice_4x4_su3_8shifts()
    b = np.zeros(p.n, dtype=np.complex128)
    res = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, b, p.sigma, p.tol)
    assert res.status == 0 and res.iters == 0
    assert np.all(res.x == 0)


# ----------------------------------------------------------------------------
# Generic block-CSR operator
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("bd", [1, 2, 3])
def test_bsr_apply_and_solve_match_dense(bd):
    rp, ci, vals, A = inputs.random_hpd_bsr(40, bd, 4, 0.5, 21 + bd)
    n = A.shape[0]
    v = _vec(n, 7)
    y = oracle.bsr_apply(rp, ci, vals, v, sigma=0.25)
    assert np.linalg.norm(y - (A @ v + 0.25 * v)) <= 1e-13 * np.linalg.norm(y)
    sig = inputs.log_shifts(1e-3, 2.0, 5)
    res = oracle.cgm_bsr(rp, ci, vals, v, sig, 1e-13)
    assert res.status == 0
    for i, s in enumerate(sig):
        xs = np.linalg.solve(A + s * np.eye(n), v)
        assert np.linalg.norm(res.x[i] - xs) <= 1e-10 * np.linalg.norm(xs)


def _dst_solve(N, b, sigma):
    """(A + sigma)^{-1} b for the N x N Dirichlet five-point Laplacian by its
    eigenbasis: sin(pi k x / (N+1)) modes, eigenvalues
    4 - 2 cos(pi k/(N+1)) - 2 cos(pi l/(N+1)) (orthonormal DST-I)."""
    from scipy.fft import dstn, idstn
    k = np.arange(1, N + 1)
    lam1 = 2.0 - 2.0 * np.cos(np.pi * k / (N + 1))
    lam = lam1[None, :] + lam1[:, None]          # [j][i] for grid row i + N j
    B = b.reshape(N, N)
    out = []
    for s in sigma:
        out.append(idstn(dstn(B, type=1, norm="ortho") / (lam + s), type=1, norm="ortho").reshape(-1))
    return np.array(out)


def test_poisson_operator_modes_and_solve_closed_form():
    N = 12
    rp, ci, va = inputs.poisson_5pt_bsr(N)
    assert rp[-1] == 5 * N * N - 4 * N           # interior 5, edges 4, corners 3
    # the sine modes are eigenvectors with the closed-form eigenvalues
    x = np.arange(1, N + 1)
    for (kx, ky) in [(1, 1), (3, 7), (N, 2)]:
        v = np.outer(np.sin(np.pi * ky * x / (N + 1)), np.sin(np.pi * kx * x / (N + 1))).reshape(-1)
        lam = 4 - 2 * np.cos(np.pi * kx / (N + 1)) - 2 * np.cos(np.pi * ky / (N + 1))
        Av = oracle.bsr_apply(rp, ci, va, v.astype(np.complex128))
        assert np.linalg.norm(Av - lam * v) <= 1e-13 * np.linalg.norm(lam * v)
    # CG-M on the paper's operator against the spectral solution
    b = _vec(N * N, 9)
    sig = inputs.log_shifts(1e-4, 10.0, 15)
    res = oracle.cgm_bsr(rp, ci, va, b, sig, 1e-13)
    assert res.status == 0
    want = _dst_solve(N, b.real, sig) + 1j * _dst_solve(N, b.imag, sig)
    for s in range(len(sig)):
        assert np.linalg.norm(res.x[s] - want[s]) <= 1e-10 * np.linalg.norm(want[s])


def test_bsr_not_hpd_is_reported():
    rp, ci, vals, A = inputs.random_hpd_bsr(10, 2, 3, 0.5, 31)
    neg = vals.copy()
    for i in range(10):
        for k in range(rp[i], rp[i + 1]):
            if ci[k] == i:
                neg[k] = -10.0 * np.eye(2) - np.abs(neg[k]).max() * np.eye(2) * 5
    v = _vec(20, 8)
    res = oracle.cgm_bsr(rp, ci, neg, v, [0.1], 1e-10, max_iter=50)
    assert res.status in (4, 6)
    # a matrix whose diagonal is strongly negative has v^dag A v < 0 at the
    # first direction p = b for this v
    Av = oracle.bsr_apply(rp, ci, neg, v)
    if np.vdot(v, Av).real < 0:
        assert res.status == 4


# ----------------------------------------------------------------------------
# Link force of S = sum_s c_s phi^dagger (A + sigma_s)^{-1} phi
# ----------------------------------------------------------------------------

def _fd_entry(U, dims, nc, m, phi, sig, c, mu, site, a, b, h, imag):
    """Central difference of S in one link entry, written without cancellation:
    S(U+) - S(U-) = sum_s c_s x_s+^dagger (A- - A+) x_s- for Hermitian A."""
    Upl = U.copy(); Umi = U.copy()
    d = (1j if imag else 1.0) * h
    Upl[mu, site, a, b] += d
    Umi[mu, site, a, b] -= d
    rp = oracle.cgm_staggered(Upl, dims, nc, m, phi, sig, 1e-13)
    rm = oracle.cgm_staggered(Umi, dims, nc, m, phi, sig, 1e-13)
    tot = 0.0
    for s in range(len(sig)):
        dA = (oracle.staggered_apply(Umi, dims, nc, m, rm.x[s])
              - oracle.staggered_apply(Upl, dims, nc, m, rm.x[s]))
        tot += c[s] * np.vdot(rp.x[s], dA).real
    return tot / (2 * h)


def test_link_force_matches_central_differences():
    dims, nc, m = (4, 4, 4, 4), 3, 0.2
    U = inputs.su_n_links(dims, nc, 0.7, 41)
    n = inputs.volume(dims) * nc
    phi = _vec(n, 9)
    sig = inputs.log_shifts(1e-2, 2.0, 4)
    c = sig ** 0.5 / 4
    res = oracle.cgm_staggered(U, dims, nc, m, phi, sig, 1e-13)
    G = oracle.link_force(U, dims, nc, c, res.x)
    g = inputs.rng(42)
    V = inputs.volume(dims)
    for _ in range(6):
        mu, site = int(g.integers(4)), int(g.integers(V))
        a, b = int(g.integers(nc)), int(g.integers(nc))
        fre = _fd_entry(U, dims, nc, m, phi, sig, c, mu, site, a, b, 1e-6, False)
        fim = _fd_entry(U, dims, nc, m, phi, sig, c, mu, site, a, b, 1e-6, True)
        got = G[mu, site, a, b]
        scale = max(abs(got), 1e-3)
        assert abs(got.real - fre) <= 1e-6 * scale, (got, fre)
        assert abs(got.imag - fim) <= 1e-6 * scale, (got, fim)


def test_phi_gradient_closed_form():
    """dS/dphi (torch convention dS/dRe + i dS/dIm) = 2 sum_s c_s x_s, checked
    by central differences on S itself for a small lattice."""
    dims, nc, m = (4, 4, 2, 2), 2, 0.3
    U = inputs.su_n_links(dims, nc, 0.5, 43)
    n = inputs.volume(dims) * nc
    phi = _vec(n, 10)
    sig = np.array([0.05, 0.5])
    c = np.array([0.7, 0.3])
    res = oracle.cgm_staggered(U, dims, nc, m, phi, sig, 1e-14)
    grad = 2 * sum(c[s] * res.x[s] for s in range(2))
    h = 1e-5
    for j in (0, 7, 33):
        for d in (1.0, 1j):
            pp = phi.copy(); pm = phi.copy()
            pp[j] += d * h; pm[j] -= d * h
            sp = oracle.quad_form(pp, oracle.cgm_staggered(U, dims, nc, m, pp, sig, 1e-14).x, c)
            sm = oracle.quad_form(pm, oracle.cgm_staggered(U, dims, nc, m, pm, sig, 1e-14).x, c)
            fd = (sp - sm) / (2 * h)
            want = grad[j].real if d == 1.0 else grad[j].imag
            assert abs(fd - want) <= 1e-6 * max(1.0, abs(want))


# ----------------------------------------------------------------------------
# BiCGStab-M: the multi-shift BiCGStab for non-Hermitian families
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("bd", [1, 2, 3])
def test_bicgstabm_matches_dense_solves(bd):
    rp, ci, va, A = inputs.random_nonhermitian_bsr(24, bd, 4, 0.5, 0.3, 40 + bd)
    assert np.linalg.norm(A - np.conj(A.T)) > 0.1 * np.linalg.norm(A)   # truly non-Hermitian
    n = A.shape[0]
    b = _vec(n, 41)
    sig = inputs.log_shifts(1e-2, 3.0, 6)
    res = oracle.bicgstabm_bsr(rp, ci, va, b, sig, 1e-13)
    assert res.status == 0
    for s, sv in enumerate(sig):
        xd = np.linalg.solve(A + sv * np.eye(n), b)
        assert np.linalg.norm(res.x[s] - xd) <= 1e-10 * np.linalg.norm(xd), (s, sv)


def test_bicgstabm_shifted_residuals_are_collinear():
    """At every iteration b - (A + sigma) x_sigma = (zeta_sigma / T_sigma) r:
    a dropped term or a wrong factor in any shifted recurrence breaks this."""
    rp, ci, va, A = inputs.random_nonhermitian_bsr(30, 2, 4, 0.5, 0.3, 51)
    n = A.shape[0]
    b = _vec(n, 52)
    sig = np.array([0.0, 0.02, 0.3, 2.0])
    for k in (1, 2, 5, 9):
        res = oracle.bicgstabm_bsr(rp, ci, va, b, sig, 0.0, max_iter=k, freeze=False)
        assert res.iters == k
        for s, sv in enumerate(sig):
            true_r = b - (A @ res.x[s] + sv * res.x[s])
            assert np.linalg.norm(true_r - res.c[s] * res.r) <= 1e-11 * np.linalg.norm(b), (k, s)
    # the seed's own first step is the textbook one: x = alpha b + omega s
    res = oracle.bicgstabm_bsr(rp, ci, va, b, [0.0], 0.0, max_iter=1, freeze=False)
    v = A @ b
    alpha = np.vdot(b, b) / np.vdot(b, v)
    s1 = b - alpha * v
    t = A @ s1
    omega = np.vdot(t, s1) / np.vdot(t, t)
    assert np.linalg.norm(res.x[0] - (alpha * b + omega * s1)) <= 1e-13 * np.linalg.norm(res.x[0])


def test_bicgstabm_dirac_family_equals_cgm_on_normal_equations():
    """(m_s + D) x = b has x = (m_s - D) y with y = (m_s^2 - D^2)^{-1} b, the
    CG-M family of A = m^2 - D^2 at shifts m_s^2 - m^2: two different
    algorithms on two different operators must agree."""
    dims, nc, m = (4, 4, 4, 6), 3, 0.1
    U = inputs.su_n_links(dims, nc, 0.6, 61)
    n = inputs.volume(dims) * nc
    b = _vec(n, 62)
    sig = inputs.log_shifts(1e-3, 1.0, 5)
    res = oracle.bicgstabm_dirac(U, dims, nc, m, b, sig, 1e-13)
    assert res.status == 0
    ms = m + sig
    y = oracle.cgm_staggered(U, dims, nc, m, b, ms ** 2 - m ** 2, 1e-13)
    assert y.status == 0
    for s in range(len(sig)):
        want = ms[s] * y.x[s] - oracle.dslash(U, dims, nc, y.x[s])
        assert np.linalg.norm(res.x[s] - want) <= 1e-9 * np.linalg.norm(want), s
        r = b - oracle.dirac_apply(U, dims, nc, m, res.x[s], sigma=sig[s])
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)


def test_staggered_dirac_bsr_matches_oracle_operator():
    dims, nc, m = (4, 2, 4, 6), 2, 0.3
    U = inputs.su_n_links(dims, nc, 0.7, 71)
    rp, ci, va = inputs.staggered_dirac_bsr(U, dims, nc, m)
    n = inputs.volume(dims) * nc
    v = _vec(n, 72)
    got = oracle.bsr_apply(rp, ci, va, v, sigma=0.25)
    want = oracle.dirac_apply(U, dims, nc, m, v, sigma=0.25)
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)


def test_bicgstabm_zero_source():
    rp, ci, va, A = inputs.random_nonhermitian_bsr(10, 3, 3, 0.5, 0.3, 81)
    res = oracle.bicgstabm_bsr(rp, ci, va, np.zeros(30, np.complex128), [0.1, 1.0], 1e-10)
    assert res.status == 0 and res.iters == 0 and np.all(res.x == 0)


def _skew_bsr(nbr):
    """A real skew-symmetric tridiagonal matrix as 1x1 block-CSR: for any real
    b, b^T A b = 0, so BiCGStab's first (r~, A p) = b^T A b vanishes."""
    rp, ci, va = [0], [], []
    for i in range(nbr):
        if i > 0:
            ci.append(i - 1); va.append(-1.0)
        if i < nbr - 1:
            ci.append(i + 1); va.append(1.0)
        rp.append(len(ci))
    return (np.asarray(rp, np.int64), np.asarray(ci, np.int32),
            np.asarray(va, np.complex128).reshape(-1, 1, 1))


def test_bicgstabm_breakdown_is_reported():
    rp, ci, va = _skew_bsr(16)
    b = np.arange(1, 17, dtype=np.float64).astype(np.complex128)
    res = oracle.bicgstabm_bsr(rp, ci, va, b, [0.0], 1e-10)
    assert res.status == 7      # breakdown


# ----------------------------------------------------------------------------
# Different right-hand side per shift, b_s = q_s(A) b (Sec. 5, eq. linprobgen)
# ----------------------------------------------------------------------------

def _poly_coefs(S, deg, seed):
    g = inputs.rng(seed)
    return g.uniform(-1.0, 1.0, size=(S, deg + 1))


def test_poly_rhs_matches_dense_solves():
    """x_s = (A + sigma_s)^{-1} q_s(A) b against LAPACK, with q_s(A) formed
    from dense matrix powers (not Horner's rule)."""
    dims, nc, m = (2, 4, 2, 4), 2, 0.2
    U = inputs.su_n_links(dims, nc, 0.6, 17)
    A = _dense_A(U, dims, nc, m)
    n = A.shape[0]
    b = _vec(n, 18)
    sig = np.array([0.0, 0.01, 0.5, 3.0])
    coef = _poly_coefs(len(sig), 3, 19)
    x, bs = oracle.solve_poly_rhs_staggered(U, dims, nc, m, b, sig, coef, 1e-13)
    for s in range(len(sig)):
        Q = sum(coef[s, k] * np.linalg.matrix_power(A, k) for k in range(coef.shape[1]))
        want_b = Q @ b
        assert np.linalg.norm(bs[s] - want_b) <= 1e-12 * np.linalg.norm(want_b)
        want = np.linalg.solve(A + sig[s] * np.eye(n), want_b)
        assert np.linalg.norm(x[s] - want) <= 1e-10 * np.linalg.norm(want)


def test_poly_rhs_constant_polynomials_reduce_to_cgm():
    """q_s = c_s (degree 0) gives c_s times the one-source CG-M solution."""
    p = inputs.lattice_4x4_su3_8shifts()
    c = np.linspace(0.5, 2.0, len(p.sigma))[:, None]
    x, _ = oracle.solve_poly_rhs_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, c, 1e-13)
    ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[0], p.sigma, 1e-13)
    for s in range(len(p.sigma)):
        want = c[s, 0] * ref.x[s]
        assert np.linalg.norm(x[s] - want) <= 1e-10 * np.linalg.norm(want)


def test_poly_rhs_division_gives_collinear_initial_residuals():
    """The construction the GPU path uses: dividing q_s(t) by (t + sigma_s)
    gives q_s(t) = q_s(-sigma_s) + (t + sigma_s) s_s(t), so the initial guess
    x_s0 = s_s(A) b leaves the residual b_s - (A + sigma_s) x_s0 =
    q_s(-sigma_s) b, collinear with b for every shift (one CG-M sequence on b
    then serves all shifts). Checked with numpy's polynomial division and the
    oracle's operator."""
    p = inputs.lattice_4x4_su3_8shifts()
    coef = _poly_coefs(len(p.sigma), 4, 20)
    b = p.b[0]
    for s, sg in enumerate(p.sigma):
        quo, rem = np.polynomial.polynomial.polydiv(coef[s], [sg, 1.0])
        c = np.polynomial.polynomial.polyval(-sg, coef[s])
        assert abs(rem[0] - c) <= 1e-13 * max(1.0, abs(c))
        x0 = oracle.poly_apply_staggered(p.links, p.dims, p.nc, p.mass, quo, b)
        bs = oracle.poly_apply_staggered(p.links, p.dims, p.nc, p.mass, coef[s], b)
        r0 = bs - oracle.staggered_apply(p.links, p.dims, p.nc, p.mass, x0, sigma=sg)
        assert np.linalg.norm(r0 - c * b) <= 1e-12 * np.linalg.norm(bs)


# ----------------------------------------------------------------------------
# Parity: A = m^2 - D^2 couples no even site to an odd one
# ----------------------------------------------------------------------------

def _site_parity(dims):
    V = inputs.volume(dims)
    x = np.arange(V)
    c0 = x % dims[0]
    c1 = (x // dims[0]) % dims[1]
    c2 = (x // (dims[0] * dims[1])) % dims[2]
    c3 = x // (dims[0] * dims[1] * dims[2])
    return (c0 + c1 + c2 + c3) & 1


@pytest.mark.parametrize("par", [0, 1])
def test_parity_sources_stay_on_their_parity(par):
    """D maps one parity to the other, so A maps a parity-p vector to a
    parity-p vector and the CG-M solution of a parity-p source is zero on the
    other parity: the reduced solve of that parity alone is exact. The sites
    of one parity, in site order, are exactly the sites x with index x // 2
    (one per pair (2k, 2k+1) along x0)."""
    dims, nc, m = (4, 6, 4, 4), 3, 0.15
    U = inputs.su_n_links(dims, nc, 0.7, 21)
    P = _site_parity(dims)
    sites = np.nonzero(P == par)[0]
    assert np.array_equal(sites // 2, np.arange(len(sites)))
    mask = np.repeat(P == par, nc)
    v = _vec(inputs.volume(dims) * nc, 22) * mask
    Dv = oracle.dslash(U, dims, nc, v)
    assert np.all(Dv[mask] == 0)
    Av = oracle.staggered_apply(U, dims, nc, m, v, sigma=0.3)
    assert np.all(Av[~mask] == 0)
    res = oracle.cgm_staggered(U, dims, nc, m, v, [0.0, 0.1, 1.0], 1e-12)
    assert res.status == 0
    assert np.all(res.x[:, ~mask] == 0)
