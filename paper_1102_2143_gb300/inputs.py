"""Seeded synthetic inputs for the shifted-family solve (A + sigma_s) x_s = b.

This module draws the seeded inputs: gauge links, sources, shift lists and
generic Hermitian positive-definite block-sparse test matrices. It holds none
of the solver's arithmetic (no Krylov step, recurrence or residual) and
imports nothing from the CUDA library or from the oracle, so both sides can be
fed the same inputs. Two functions assemble an operator as block-CSR input
for the generic path: the paper's five-point Poisson matrix
(`poisson_5pt_bsr`) and the staggered Dirac matrix m + D (`staggered_dirac_bsr`);
both are checked against the oracle's own operators in the CPU tests.

Conventions (shared by every consumer of these arrays):
  * lattice dims = (L0, L1, L2, L3); site = x0 + L0*(x1 + L1*(x2 + L2*x3)),
    x0 fastest;
  * links have shape [4][V][Nc][Nc], complex128, U[mu][site][a][b];
  * a colour vector has shape [V*Nc], complex128, index = site*Nc + colour;
  * several right-hand sides stack as [nrhs][V*Nc].

The paper's application is the shifted family of eq. (linprob) (Sec. 2) with
a lattice-gauge operator; the staggered operator and the SU(N) link
distribution used here are the synthetic workload, not something the paper
fixes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def su_n_links(dims, nc: int, eps: float, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Links U = exp(i*eps*H), H a random traceless Hermitian Nc x Nc matrix.

    H = (G + G^dagger)/2 - tr(.)/Nc with G's entries complex normal
    (real and imaginary parts ~ N(0, 1/2)); the exponential is taken through
    the eigendecomposition of H, so U is unitary with det U = 1 to rounding.
    eps = 0 gives the free field U = 1.
    """
    V = volume(dims)
    if eps == 0.0:
        return np.broadcast_to(np.eye(nc, dtype=np.complex128), (4, V, nc, nc)).copy()
    g = rng(seed)
    total = 4 * V
    out = np.empty((total, nc, nc), dtype=np.complex128)
    eye = np.eye(nc)
    for lo in range(0, total, chunk):
        hi = min(total, lo + chunk)
        m = hi - lo
        G = (g.standard_normal((m, nc, nc)) + 1j * g.standard_normal((m, nc, nc))) * math.sqrt(0.5)
        H = 0.5 * (G + np.conj(np.swapaxes(G, 1, 2)))
        tr = np.trace(H, axis1=1, axis2=2).real / nc
        H = H - tr[:, None, None] * eye
        w, Q = np.linalg.eigh(H)
        ph = np.exp(1j * eps * w)
        out[lo:hi] = (Q * ph[:, None, :]) @ np.conj(np.swapaxes(Q, 1, 2))
    return out.reshape(4, V, nc, nc)


def gaussian_source(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian vector(s), real and imaginary parts ~ N(0, 1/2)."""
    g = rng(seed)
    shape = (n,) if nrhs is None else (nrhs, n)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * math.sqrt(0.5)


def log_shifts(lo: float, hi: float, count: int) -> np.ndarray:
    """`count` shifts log-spaced from lo to hi, both endpoints included."""
    if count == 1:
        return np.array([lo], dtype=np.float64)
    return np.logspace(math.log10(lo), math.log10(hi), count).astype(np.float64)


def random_gauge(dims, nc: int, seed: int) -> np.ndarray:
    """Random SU(Nc) matrices g(x), one per site, shape [V][Nc][Nc]."""
    return _random_unitary(volume(dims), nc, seed)


def _random_unitary(count: int, nc: int, seed: int) -> np.ndarray:
    g = rng(seed)
    G = (g.standard_normal((count, nc, nc)) + 1j * g.standard_normal((count, nc, nc))) * math.sqrt(0.5)
    H = 0.5 * (G + np.conj(np.swapaxes(G, 1, 2)))
    H = H - (np.trace(H, axis1=1, axis2=2).real / nc)[:, None, None] * np.eye(nc)
    w, Q = np.linalg.eigh(H)
    return (Q * np.exp(2.0j * w)[:, None, :]) @ np.conj(np.swapaxes(Q, 1, 2))


def random_hpd_bsr(nbr: int, bd: int, blocks_per_row: int, shift: float, seed: int):
    """A random Hermitian positive-definite matrix in block-CSR form.

    A = B^dagger B + shift*I where B has `blocks_per_row` random complex blocks
    per block row at random block columns (the diagonal block always present),
    so the pattern of A is ragged. Returns (row_ptr int64 [nbr+1],
    col_idx int32 [nnzb], vals complex128 [nnzb][bd][bd]) with block columns
    sorted inside each row. Intended for small test sizes (dense assembly).
    """
    g = rng(seed)
    n = nbr * bd
    B = np.zeros((n, n), dtype=np.complex128)
    for i in range(nbr):
        cols = set([i])
        k = int(g.integers(1, blocks_per_row + 1))
        while len(cols) < min(k, nbr):
            cols.add(int(g.integers(0, nbr)))
        for j in cols:
            blk = (g.standard_normal((bd, bd)) + 1j * g.standard_normal((bd, bd))) * math.sqrt(0.5)
            B[i * bd:(i + 1) * bd, j * bd:(j + 1) * bd] = blk
    A = np.conj(B.T) @ B + shift * np.eye(n)
    A = 0.5 * (A + np.conj(A.T))
    row_ptr = [0]
    cols_all = []
    vals = []
    for i in range(nbr):
        for j in range(nbr):
            blk = A[i * bd:(i + 1) * bd, j * bd:(j + 1) * bd]
            if np.any(blk != 0):
                cols_all.append(j)
                vals.append(blk)
        row_ptr.append(len(cols_all))
    return (np.asarray(row_ptr, dtype=np.int64), np.asarray(cols_all, dtype=np.int32),
            np.asarray(vals, dtype=np.complex128).reshape(-1, bd, bd), A)


def poisson_5pt_bsr(N: int):
    """The 2-D Poisson operator of Sec. 4: the five-point finite-difference
    Laplacian on an N x N grid (Dirichlet boundaries, unit spacing), as
    block-CSR with 1 x 1 blocks. Grid point (i, j) -> row i + N j; A has 4 on
    the diagonal and -1 for each of the up to four grid neighbours, columns
    sorted inside a row. It is real symmetric positive definite; values are
    returned as complex128 (imaginary parts zero) for the complex solver.
    Returns (row_ptr int64 [N*N+1], col_idx int32 [nnz], vals [nnz][1][1]).
    """
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    i, j = idx % N, idx // N
    # neighbours in column order: (i, j-1), (i-1, j), self, (i+1, j), (i, j+1)
    cand = [(idx - N, j > 0, -1.0), (idx - 1, i > 0, -1.0), (idx, np.ones(n, bool), 4.0),
            (idx + 1, i < N - 1, -1.0), (idx + N, j < N - 1, -1.0)]
    cols = np.stack([c for c, _, _ in cand], axis=1)
    mask = np.stack([m for _, m, _ in cand], axis=1)
    vals = np.broadcast_to(np.array([v for _, _, v in cand]), (n, 5))
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[mask].astype(np.int32)
    v = vals[mask].astype(np.complex128).reshape(-1, 1, 1)
    return row_ptr, col_idx, v


def random_nonhermitian_bsr(nbr: int, bd: int, blocks_per_row: int, shift: float, skew: float, seed: int):
    """A random non-Hermitian block-CSR matrix: the Hermitian positive-definite
    B^dagger B + shift*I of random_hpd_bsr plus `skew` times independent
    complex Gaussian blocks on the same pattern (so the field of values stays
    in the right half plane for small skew). Returns (row_ptr, col_idx, vals,
    dense A)."""
    rp, ci, va, _ = random_hpd_bsr(nbr, bd, blocks_per_row, shift, seed)
    g = rng(seed + 1)
    va = va + skew * (g.standard_normal(va.shape) + 1j * g.standard_normal(va.shape)) * math.sqrt(0.5)
    n = nbr * bd
    A = np.zeros((n, n), dtype=np.complex128)
    for i in range(nbr):
        for k in range(rp[i], rp[i + 1]):
            j = int(ci[k])
            A[i * bd:(i + 1) * bd, j * bd:(j + 1) * bd] += va[k]
    return rp, ci, va, A


def staggered_dirac_bsr(links, dims, nc: int, mass: float):
    """The staggered Dirac operator M = m + D as block-CSR with nc x nc blocks:
    per site row the diagonal m*I and, per direction mu, the forward hop
    +1/2 eta_mu(x) U_mu(x) (column x+mu) and the backward hop
    -1/2 eta_mu(x) U_mu(x-mu)^dagger (column x-mu), columns sorted; hops that
    land on the same site (extent 2) add. Conventions as in the module
    docstring. Returns (row_ptr int64, col_idx int32, vals [nnzb][nc][nc])."""
    dims = tuple(int(d) for d in dims)
    V = volume(dims)
    U = np.asarray(links, dtype=np.complex128).reshape(4, V, nc, nc)
    x = np.arange(V)
    c = [(x // int(np.prod(dims[:mu]))) % dims[mu] for mu in range(4)]
    stride = [int(np.prod(dims[:mu])) for mu in range(4)]
    cols = [x]
    blks = [np.broadcast_to(mass * np.eye(nc, dtype=np.complex128), (V, nc, nc))]
    for mu in range(4):
        par = sum(c[nu] for nu in range(mu)) if mu else np.zeros(V, dtype=np.int64)
        eta = np.where(par % 2 == 0, 0.5, -0.5)[:, None, None]
        fwd = np.where(c[mu] == dims[mu] - 1, x - (dims[mu] - 1) * stride[mu], x + stride[mu])
        bwd = np.where(c[mu] == 0, x + (dims[mu] - 1) * stride[mu], x - stride[mu])
        cols += [fwd, bwd]
        blks += [eta * U[mu], -eta * np.conj(np.swapaxes(U[mu][bwd], 1, 2))]
    cols = np.stack(cols, axis=1)                     # [V][9]
    blks = np.stack(blks, axis=1)                     # [V][9][nc][nc]
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    blks = np.take_along_axis(blks, order[:, :, None, None], axis=1)
    if min(dims) > 2:       # no two hops of a row land on the same site
        return (np.arange(V + 1, dtype=np.int64) * 9, cols.reshape(-1).astype(np.int32),
                np.ascontiguousarray(blks.reshape(-1, nc, nc)))
    # merge repeated columns inside a row
    row_ptr = [0]
    out_c, out_b = [], []
    for i in range(V):
        prev = -1
        for k in range(9):
            if cols[i, k] == prev:
                out_b[-1] = out_b[-1] + blks[i, k]
            else:
                out_c.append(cols[i, k])
                out_b.append(blks[i, k].copy())
                prev = cols[i, k]
        row_ptr.append(len(out_c))
    return (np.asarray(row_ptr, dtype=np.int64), np.asarray(out_c, dtype=np.int32),
            np.asarray(out_b, dtype=np.complex128))


@dataclass
class PoissonProblem:
    """The shifted family on the 2-D Poisson operator (the paper's test)."""
    N: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray
    b: np.ndarray        # [n] complex128
    sigma: np.ndarray    # [S]
    tol: float

    @property
    def n(self) -> int:
        return self.N * self.N


def poisson_2d_15shifts(N: int = 1000, seed_base: int = 5000) -> PoissonProblem:
    """N x N five-point Poisson operator, 15 shifts log-spaced 1e-4..10, a
    complex Gaussian source (seed_base+1), tol 1e-10. The paper names 15
    shifts and the 1000 x 1000 grid but not the shift values or the source."""
    rp, ci, va = poisson_5pt_bsr(N)
    b = gaussian_source(N * N, seed_base + 1)
    return PoissonProblem(N, rp, ci, va, b, log_shifts(1e-4, 10.0, 15), 1e-10)


@dataclass
class StaggeredProblem:
    """One synthetic staggered shifted-family problem."""
    dims: tuple
    nc: int
    mass: float
    eps: float
    links: np.ndarray      # [4][V][Nc][Nc] complex128
    b: np.ndarray          # [nrhs][V*Nc] complex128
    sigma: np.ndarray      # [S] float64
    tol: float

    @property
    def n(self) -> int:
        return volume(self.dims) * self.nc


def staggered_problem(L, nc, mass, eps, shifts, nrhs, tol, seed_base) -> StaggeredProblem:
    """Links from seed_base+0, sources from seed_base+1."""
    dims = (L, L, L, L) if np.isscalar(L) else tuple(L)
    links = su_n_links(dims, nc, eps, seed_base + 0)
    b = gaussian_source(volume(dims) * nc, seed_base + 1, nrhs)
    return StaggeredProblem(dims, nc, float(mass), float(eps), links, b,
                            np.asarray(shifts, dtype=np.float64), float(tol))


# The five synthetic workloads, named by what they are.
def lattice_4x4_su3_8shifts(nrhs: int = 1) -> StaggeredProblem:
    """4^4 SU(3), eps=0.5, m=0.1, 8 shifts log-spaced 1e-3..1, tol 1e-10."""
    return staggered_problem(4, 3, 0.1, 0.5, log_shifts(1e-3, 1.0, 8), nrhs, 1e-10, 0)


def lattice_24x4_su3_15shifts(L: int = 24, nrhs: int = 1) -> StaggeredProblem:
    """24^4 SU(3), eps=0.8, m=0.05, 15 shifts log-spaced 1e-4..10, tol 1e-10.

    Exported as block-CSR (3x3 complex blocks) for the generic path. `L` lets
    tests build the same recipe on a smaller lattice.
    """
    return staggered_problem(L, 3, 0.05, 0.8, log_shifts(1e-4, 10.0, 15), nrhs, 1e-10, 1000)


def lattice_16x4_su3_force(L: int = 16):
    """16^4 SU(3), eps=0.7, m=0.05; 12 (sigma_s, c_s) with sigma log-spaced
    1e-4..5 and c_s = sigma_s**0.5 / 12; Gaussian phi."""
    sig = log_shifts(1e-4, 5.0, 12)
    c = sig ** 0.5 / 12.0
    p = staggered_problem(L, 3, 0.05, 0.7, sig, 1, 1e-10, 3000)
    return p, c


def lattice_32x4_su3_20shifts(L: int = 32, nrhs: int = 8) -> StaggeredProblem:
    """32^4 SU(3), eps=0.9, m=0.01, 20 shifts log-spaced 1e-5..10, 8 RHS."""
    return staggered_problem(L, 3, 0.01, 0.9, log_shifts(1e-5, 10.0, 20), nrhs, 1e-10, 4000)


def batched_uneven_systems(count: int = 64, seed_base: int = 2000):
    """`count` independent staggered problems: L from {4,6,8,10,12}, SU(2) or
    SU(3), m ~ U[0.02, 0.2], eps = 0.6, S ~ U{4..20} shifts log-spaced
    1e-4..1, 4 Gaussian right-hand sides each."""
    g = rng(seed_base + 2)
    out = []
    for i in range(count):
        L = int(g.choice([4, 6, 8, 10, 12]))
        nc = int(g.choice([2, 3]))
        m = float(g.uniform(0.02, 0.2))
        S = int(g.integers(4, 21))
        out.append(staggered_problem(L, nc, m, 0.6, log_shifts(1e-4, 1.0, S), 4, 1e-10,
                                     seed_base + 10 * (i + 1)))
    return out
