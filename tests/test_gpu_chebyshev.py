"""GPU parity of the Chebyshev smoother option (smoother = 1: point-block-Jacobi-preconditioned
Chebyshev acceleration of degree cheb_degree on [0.1, 1.1] x lambda_max(D^-1 A) per level),
called through the C ABI, against the oracle's V-cycle and direct solve on the same seeded
inputs.  Bounds as for the Jacobi smoother: FP64 cycle 1e-9 relative (the power-iteration
estimate of lambda and the recurrence differ only in rounding order), FP32 cycle 1e-3, solves
1e-8 true relative residual and 1e-6 displacement / compliance error."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, mg, solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


CHEB = dict(smoother="chebyshev")


@pytest.mark.parametrize("pc,kw,okw", [
    ("gmg", dict(n_levels=3), dict(n_levels=3)),
    ("amg", dict(max_coarse_dofs=80), dict(cap=80)),
    ("hybrid", dict(n_geo_levels=2, max_coarse_dofs=80), dict(n_geo=2, cap=80))])
@pytest.mark.parametrize("dim,grid", [(2, (30, 14, 1)), (3, (8, 6, 5))])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_vcycle_chebyshev(lib, ctx, pc, kw, okw, dim, grid, m):
    p = W.random_problem(dim, *grid, seed=13, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc=pc, prec="fp64", smoother="chebyshev", cheb_degree=m, **kw)
    H = osolve.build(p, pc=pc, smoother="chebyshev", cheb_degree=m, **okw)
    assert P.num_levels() == H.n_levels
    r = np.random.default_rng(1).standard_normal(p.n)
    zr = mg.vcycle(H, r)
    assert relerr(P.vcycle(r), zr) < 1e-9
    P.setup(pc=pc, prec="fp32", smoother="chebyshev", cheb_degree=m, **kw)
    assert relerr(P.vcycle(r), zr) < 1e-3
    if dim == 3:
        P.setup(pc=pc, prec="tc", smoother="chebyshev", cheb_degree=m, **kw)
        assert relerr(P.vcycle(r), zr) < 1e-3


@pytest.mark.parametrize("pc,kw,okw", [
    ("gmg", dict(n_levels=4), dict(n_levels=4)),
    ("hybrid", dict(n_geo_levels=2, max_coarse_dofs=200), dict(n_geo=2, cap=200))])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc"])
@pytest.mark.parametrize("case", ["mbb", "cant2d", "cant3d"])
def test_solve_chebyshev_vs_direct(lib, ctx, pc, kw, okw, prec, case):
    if case == "mbb":
        p = W.mbb_beam(96, 32)
    elif case == "cant2d":
        p = W.cantilever_2d(96, 48, seed=0, sigma=4.0)
    else:
        p = W.cantilever_3d(16, 8, 8, seed=0, sigma=2.0)
        if pc == "gmg":
            kw, okw = dict(n_levels=3), dict(n_levels=3)
    if prec == "tc" and case != "cant3d":
        pytest.skip("the tensor-core operator is the hex8 one")
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc=pc, prec=prec, rtol=1e-8, **CHEB, **kw)
    u, res = P.solve(p.f)
    r = res[0]
    assert r["status"] == 0, r
    ref = osolve.direct(p)
    A0 = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * p.f[0]
    assert np.linalg.norm(b - A0 @ u[0]) / np.linalg.norm(b) <= 1.05e-8
    assert r["rel_residual"] <= 1e-8
    assert relerr(u, ref["u"]) <= 1e-6
    assert abs(r["compliance"] - ref["compliance"][0]) <= 1e-6 * abs(ref["compliance"][0])
    if prec == "fp64" and pc == "gmg":
        o = osolve.solve(p, pc="gmg", smoother="chebyshev", **okw)
        oi = int(o["iterations"][0])
        slack = max(1, int(0.05 * oi)) if case == "cant2d" else 1
        assert abs(oi - r["iterations"]) <= slack


def test_chebyshev_fewer_iterations_than_jacobi(lib, ctx):
    p = W.mbb_beam(96, 32)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=4, prec="fp32")
    _, rj = P.solve(p.f)
    P.setup(pc="gmg", n_levels=4, prec="fp32", **CHEB)
    _, rc = P.solve(p.f)
    assert rc[0]["iterations"] < rj[0]["iterations"]


def test_chebyshev_invalid_options(lib, ctx):
    p = W.mbb_beam(8, 4)
    P = lib.Problem.from_workload(ctx, p)
    for bad in (dict(cheb_degree=0), dict(cheb_degree=9), dict(cheb_lower=0.0),
                dict(cheb_lower=1.2, cheb_upper=1.1)):
        with pytest.raises(lib.TomgError):
            P.setup(pc="gmg", n_levels=2, **CHEB, **bad)


def _geo_levels(P):
    """Geometric levels of the current hierarchy (levels whose transfer is geometric, + 1)."""
    n = P.num_levels()
    return 1 + sum(1 for l in range(n - 1) if P.level_info(l)["geometric"])


def test_adaptive_hybrid_drops_geometric_levels(lib, ctx):
    """Sec. 4.4: start with 6 geometric levels; every solve above the iteration limit makes the
    next setup use one fewer, down to the minimum of 2.  A limit of 3 iterations is exceeded by
    every solve here, so the sequence is 6, 5, 4, 3, 2, 2; every solve stays exact."""
    p = W.cantilever_3d(32, 16, 16, seed=0, sigma=2.0)
    P = lib.Problem.from_workload(ctx, p)
    ref = osolve.direct(p)
    seen = []
    for _ in range(6):
        P.setup(pc="hybrid", prec="fp32", n_geo_levels=6, max_coarse_dofs=1000,
                adaptive_geo=1, adaptive_iters=3, adaptive_min_geo=2)
        seen.append(_geo_levels(P))
        u, res = P.solve(p.f)
        assert res[0]["status"] == 0 and res[0]["iterations"] > 3
        assert relerr(u, ref["u"]) <= 1e-6
    assert seen == [6, 5, 4, 3, 2, 2], seen
    assert P.adaptive_geo_levels() == 2


def test_adaptive_hybrid_keeps_levels_below_limit(lib, ctx):
    p = W.cantilever_3d(16, 8, 8, seed=0, sigma=2.0)
    P = lib.Problem.from_workload(ctx, p)
    for _ in range(3):
        P.setup(pc="hybrid", prec="fp32", n_geo_levels=3, max_coarse_dofs=200, adaptive_geo=1)
        _, res = P.solve(p.f)
        assert res[0]["iterations"] <= 200
    assert P.adaptive_geo_levels() == 3


@pytest.mark.parametrize("dim,grid,prec,pc,kw", [
    (3, (16, 8, 8), "tc", "hybrid", dict(n_geo_levels=3, max_coarse_dofs=200)),
    (3, (13, 7, 9), "tc", "gmg", dict(n_levels=3)),     # odd axes: last coarse partners
    (3, (12, 6, 6), "fp64", "gmg", dict(n_levels=3)),
    (2, (64, 33, 1), "fp32", "gmg", dict(n_levels=4)),
])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_fused_transfers_bit_identical(lib, ctx, dim, grid, prec, pc, kw, m):
    """Algorithm 1 with the prolongation computed inside the first post-smoothing step (and, on
    the hex8 tensor-core level 0, the first step from x = 0 inside the second): the V-cycle and
    the whole solve are bit-identical to the cycle with separate transfer launches."""
    p = W.random_problem(dim, *grid, seed=41, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    r = np.random.default_rng(42).standard_normal(p.n)
    out = []
    for fuse in (0, 1):
        P.setup(pc=pc, prec=prec, smoother="chebyshev", cheb_degree=m, fuse_transfers=fuse, **kw)
        z = P.vcycle(r)
        u, res = P.solve(p.f)
        out.append((z, u, res[0]["iterations"], res[0]["status"]))
    (z0, u0, i0, s0), (z1, u1, i1, s1) = out
    assert s0 == 0 and s1 == 0
    assert np.array_equal(z0, z1)
    assert i0 == i1 and np.array_equal(u0, u1)
