"""The seeded synthetic workloads have the shapes, ranges and structure the
recipes state (lattice, gauge group, masses, shift lists, sources), draw the
same numbers for the same seed, and their links are special unitary."""
import numpy as np

from paper_1102_2143_gb300 import inputs


def _su_n(U, tol=1e-12):
    nc = U.shape[-1]
    M = U.reshape(-1, nc, nc)
    eye = np.eye(nc)
    unit = np.max(np.abs(M @ np.conj(np.swapaxes(M, 1, 2)) - eye))
    det = np.max(np.abs(np.linalg.det(M) - 1.0))
    return unit <= tol and det <= tol


def test_small_parity_workload():
    p = inputs.lattice_4x4_su3_8shifts()
    assert p.dims == (4, 4, 4, 4) and p.nc == 3 and p.mass == 0.1 and p.eps == 0.5
    assert p.links.shape == (4, 256, 3, 3) and p.b.shape == (1, 768)
    np.testing.assert_allclose(p.sigma, np.logspace(-3, 0, 8))
    assert p.tol == 1e-10 and _su_n(p.links)


def test_benchmark_workload_recipe_on_a_small_lattice():
    p = inputs.lattice_24x4_su3_15shifts(L=6)
    assert p.dims == (6, 6, 6, 6) and p.mass == 0.05 and p.eps == 0.8
    np.testing.assert_allclose(p.sigma, np.logspace(-4, 1, 15))
    assert _su_n(p.links)
    # complex Gaussian source: real and imaginary parts N(0, 1/2)
    b = inputs.gaussian_source(200000, 3)
    assert abs(np.var(b.real) - 0.5) < 0.01 and abs(np.var(b.imag) - 0.5) < 0.01


def test_large_and_force_recipes():
    p = inputs.lattice_32x4_su3_20shifts(L=4, nrhs=8)
    assert p.mass == 0.01 and p.eps == 0.9 and p.b.shape == (8, 768)
    np.testing.assert_allclose(p.sigma, np.logspace(-5, 1, 20))
    f, c = inputs.lattice_16x4_su3_force(L=4)
    np.testing.assert_allclose(f.sigma, np.logspace(-4, np.log10(5.0), 12))
    np.testing.assert_allclose(c, f.sigma ** 0.5 / 12.0)
    assert f.mass == 0.05 and f.eps == 0.7


def test_batched_recipe_ranges():
    probs = inputs.batched_uneven_systems(64)
    assert len(probs) == 64
    for q in probs:
        assert q.dims[0] in (4, 6, 8, 10, 12) and len(set(q.dims)) == 1
        assert q.nc in (2, 3) and 0.02 <= q.mass <= 0.2 and q.eps == 0.6
        assert 4 <= len(q.sigma) <= 20 and q.b.shape[0] == 4
        assert np.isclose(q.sigma[0], 1e-4) and np.isclose(q.sigma[-1], 1.0)
    assert {q.nc for q in probs} == {2, 3}
    assert len({q.dims[0] for q in probs}) == 5


def test_same_seed_same_numbers_and_free_field():
    a = inputs.su_n_links((4, 4, 2, 2), 2, 0.6, 11)
    b = inputs.su_n_links((4, 4, 2, 2), 2, 0.6, 11)
    c = inputs.su_n_links((4, 4, 2, 2), 2, 0.6, 12)
    assert np.array_equal(a, b) and not np.array_equal(a, c) and _su_n(a)
    assert np.array_equal(inputs.su_n_links((2, 2, 2, 2), 3, 0.0, 1),
                          np.broadcast_to(np.eye(3), (4, 16, 3, 3)))
