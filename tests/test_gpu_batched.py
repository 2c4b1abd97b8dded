"""Several right-hand sides on one hierarchy (the paper's multiple-solve setting, Sec. 2.2 / 4.2):
concurrent solve slots give the same answers as one-at-a-time solves and as the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dim,grid,pc", [(2, (48, 24, 1), "hybrid"), (3, (12, 8, 6), "gmg")])
def test_concurrent_slots_identical_to_serial(lib, ctx, dim, grid, pc):
    if dim == 2:
        p = W.random_problem(2, *grid, seed=31, contrast="minmax", nrhs=7)
    else:
        p = W.batched_3d(*grid, n_loads=3, n_adjoint=3)
    P = lib.Problem.from_workload(ctx, p)
    kw = dict(pc=pc, prec="fp32", max_coarse_dofs=150, n_geo_levels=2, n_levels=3)
    P.setup(concurrency=1, **kw)
    U1, r1 = P.solve(p.f)
    P.setup(concurrency=4, **kw)
    U4, r4 = P.solve(p.f)
    assert [r["iterations"] for r in r1] == [r["iterations"] for r in r4]
    assert np.array_equal(U1, U4)  # fixed reduction order: slot assignment does not matter
    ref = osolve.direct(p)
    for j in range(p.nrhs):
        assert r4[j]["status"] == 0 and r4[j]["rel_residual"] <= 1e-8
        assert relerr(U4[j], ref["u"][j]) <= 1e-6


def test_batched_device_arrays_and_warm_start(lib, ctx):
    import torch
    p = W.batched_3d(10, 6, 6, n_loads=4, n_adjoint=4)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=2, prec="fp32", concurrency=8)
    f = torch.tensor(p.f, dtype=torch.float64, device="cuda:0")
    U, res = P.solve(f)
    assert len(res) == 8 and all(r["status"] == 0 for r in res)
    U2, res2 = P.solve(f, u0=U)
    assert all(r["iterations"] <= 1 for r in res2)
    ref = osolve.direct(p)
    assert relerr(U.cpu().numpy(), ref["u"]) <= 1e-6


BLOCK_CASES = [("hybrid", dict(n_geo_levels=2, max_coarse_dofs=150), "chebyshev"),
               ("gmg", dict(n_levels=3), "jacobi"),
               ("amg", dict(max_coarse_dofs=150), "chebyshev")]


@pytest.mark.parametrize("pc,kw,smoother", BLOCK_CASES)
def test_block_solve_identical_to_single(lib, ctx, pc, kw, smoother):
    """The block solve (every launch covers all right-hand sides, per-right-hand-side scalars
    and convergence) gives bit-identical solutions and iteration counts to the solves one at a
    time; blocks of 4 + 3 right-hand sides, on geometric, algebraic and hybrid hierarchies."""
    p = W.batched_3d(20, 10, 10, n_loads=4, n_adjoint=3)
    P = lib.Problem.from_workload(ctx, p)
    opts = dict(pc=pc, prec="tc", smoother=smoother, cheb_degree=2, rtol=1e-8, **kw)
    P.setup(concurrency=1, **opts)
    U1, r1 = P.solve(p.f)
    P.setup(block_rhs=4, **opts)
    Ub, rb = P.solve(p.f)
    assert [r["iterations"] for r in rb] == [r["iterations"] for r in r1]
    assert np.array_equal(Ub, U1)
    ref = osolve.direct(p)
    for j in range(p.nrhs):
        assert rb[j]["status"] == 0 and rb[j]["rel_residual"] <= 1e-8
        assert relerr(Ub[j], ref["u"][j]) <= 1e-6
        assert abs(rb[j]["compliance"] - ref["compliance"][j]) <= 1e-6 * abs(ref["compliance"][j])


def test_block_solve_mixed_convergence_and_zero_rhs(lib, ctx):
    """Right-hand sides that converge at different iterations, a zero right-hand side (0
    iterations, u = 0) and a warm start that is already converged share one block."""
    p = W.batched_3d(16, 8, 8, n_loads=2, n_adjoint=2)
    f = np.concatenate([p.f, np.zeros((1, p.n))])
    P = lib.Problem.from_workload(ctx, p)
    opts = dict(pc="hybrid", n_geo_levels=2, max_coarse_dofs=150, prec="tc",
                smoother="chebyshev", rtol=1e-8)
    P.setup(concurrency=1, **opts)
    U1, r1 = P.solve(f)
    P.setup(block_rhs=8, **opts)
    Ub, rb = P.solve(f)
    assert [r["iterations"] for r in rb] == [r["iterations"] for r in r1]
    assert np.array_equal(Ub, U1)
    assert rb[-1]["iterations"] == 0 and not Ub[-1].any()
    U2, r2 = P.solve(f, u0=Ub)
    assert all(r["iterations"] <= 1 for r in r2)


def test_block_solve_rejects_unsupported(lib, ctx):
    p = W.random_problem(2, 12, 8, seed=3, contrast="minmax", nrhs=2)
    P = lib.Problem.from_workload(ctx, p)
    with pytest.raises(lib.TomgError):
        P.setup(pc="gmg", n_levels=2, prec="fp32", block_rhs=4)
