"""Batched uneven systems: many staggered problems (different lattices,
SU(2)/SU(3), shift counts, right-hand sides) solved in one batch, checked
problem by problem against the FP64 oracle: x_s within 1e-8 relative of the
oracle's solution and FP64 true residual <= 1e-10 for every shift."""
import time

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
    c = msc.msc_create(0, torch.cuda.current_stream())
    yield c
    msc.msc_destroy(c)


def mini_batch():
    spec = [((4, 4, 4, 4), 3, 0.10, 5, 2), ((6, 4, 4, 6), 2, 0.05, 8, 2),
            ((4, 6, 2, 4), 2, 0.20, 4, 1), ((6, 6, 6, 6), 3, 0.08, 11, 3),
            ((2, 4, 4, 8), 3, 0.15, 6, 2)]
    out = []
    for i, (dims, nc, m, S, nrhs) in enumerate(spec):
        out.append(inputs.staggered_problem(dims, nc, m, 0.6, inputs.log_shifts(1e-4, 1.0, S), nrhs,
                                            1e-10, 7000 + 10 * i))
    return out


def check_problem(p, x, tol=1e-10):
    for r in range(p.b.shape[0]):
        ref = oracle.cgm_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, 1e-13)
        rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, x[r])
        assert np.all(rho <= tol), rho
        for s in range(len(p.sigma)):
            assert rel(x[r][s], ref.x[s]) <= 1e-8, (r, s, rel(x[r][s], ref.x[s]))


@pytest.mark.parametrize("prec", [msc.MSC_FP64, msc.MSC_MIXED])
def test_mini_batch_against_oracle(ctx, prec):
    probs = mini_batch()
    ops = [msc.msc_op_staggered(ctx, p.nc, p.dims, p.links, p.mass) for p in probs]
    xs, infos, tun = msc.solve_batched(ctx, [(op, p.b, p.sigma) for op, p in zip(ops, probs)],
                                       precision=prec)
    for p, x, info in zip(probs, xs, infos):
        assert info.status == 0
        check_problem(p, x)
        assert np.all(info.true_rel_resid <= 1e-10)
    assert tun.site_threads in (64, 128, 256) and tun.vec_units in (1, 2, 4)
    # the same batch again reuses the tuned shape and gives the same answer
    xs2, _, tun2 = msc.solve_batched(ctx, [(op, p.b, p.sigma) for op, p in zip(ops, probs)],
                                     precision=prec)
    assert tun2.tuned == 0 and tun2.site_threads == tun.site_threads
    for a, b in zip(xs, xs2):
        assert np.array_equal(a, b)
    for op in ops:
        msc.msc_op_destroy(op)


def test_batched_equals_one_by_one(ctx):
    probs = mini_batch()[:3]
    ops = [msc.msc_op_staggered(ctx, p.nc, p.dims, p.links, p.mass) for p in probs]
    xs, _, _ = msc.solve_batched(ctx, [(op, p.b, p.sigma) for op, p in zip(ops, probs)],
                                 precision=msc.MSC_MIXED)
    for op, p, x in zip(ops, probs, xs):
        x1, _ = msc.solve(ctx, op, p.b, p.sigma, precision=msc.MSC_MIXED)
        for r in range(p.b.shape[0]):
            for s in range(len(p.sigma)):
                assert rel(x[r][s], x1[r][s]) <= 1e-8
        msc.msc_op_destroy(op)


def test_batched_rejects_foreign_and_bsr_operators(ctx):
    p = mini_batch()[0]
    other = msc.msc_create(0, None)
    op_other = msc.msc_op_staggered(other, p.nc, p.dims, p.links, p.mass)
    with pytest.raises(msc.MscError) as e:
        msc.solve_batched(ctx, [(op_other, p.b, p.sigma)])
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(op_other)
    msc.msc_destroy(other)
    rp, ci, va, A = inputs.random_hpd_bsr(8, 2, 3, 0.5, 1)
    bop = msc.msc_op_bsr(ctx, 8, 2, rp, ci, va)
    with pytest.raises(msc.MscError) as e:
        msc.solve_batched(ctx, [(bop, inputs.gaussian_source(16, 2), [0.1])])
    assert e.value.code == msc.MSC_ERR_ARG
    msc.msc_op_destroy(bop)


def test_64_uneven_systems_workload(ctx):
    """64 problems, L in {4,6,8,10,12}, SU(2) or SU(3), m in [0.02,0.2],
    eps = 0.6, 4..20 shifts 1e-4..1, 4 right-hand sides each, mixed precision.
    Every shift's FP64 true residual is recomputed by the oracle; every eighth
    problem is compared shift by shift with the oracle's solution."""
    probs = inputs.batched_uneven_systems(64)
    ops = [msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
           for p in probs]
    items = [(op, torch.from_numpy(p.b).cuda(), p.sigma) for op, p in zip(ops, probs)]
    msc.solve_batched(ctx, items)  # warm-up (tunes)
    torch.cuda.synchronize()
    t = time.perf_counter()
    xs, infos, tun = msc.solve_batched(ctx, items)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t
    t = time.perf_counter()
    for op, b, sig in items:
        msc.solve(ctx, op, b, sig)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t
    print(f"\n64 uneven systems: batched {t_batch*1e3:.1f} ms, one by one {t_seq*1e3:.1f} ms, "
          f"shape {tun.site_threads}/{tun.vec_threads}x{tun.vec_units}")
    for i, (p, x, info) in enumerate(zip(probs, xs, infos)):
        assert info.status == 0
        xh = x.cpu().numpy()
        for r in range(p.b.shape[0]):
            rho = oracle.true_residual_staggered(p.links, p.dims, p.nc, p.mass, p.b[r], p.sigma, xh[r])
            assert np.all(rho <= 1e-10), (i, r, rho.max())
        if i % 8 == 0:
            check_problem(p, xh)
    assert t_batch < t_seq
    for op in ops:
        msc.msc_op_destroy(op)
