"""GPU solutions at the full benchmark sizes against the oracle's reference solutions.

The references (tests/golden/*.txt, written by tests/golden/make_large_golden.py from the
oracle alone) are the solution of K(rho) u = f (Sec. 3.1): the oracle's refined sparse direct
solve for the 2D workloads, and for the 3D workloads, too large for a direct solve on a host,
the oracle's FP64 PCG to a true relative residual of about 1e-12, confirmed by a second solve
with a different preconditioner (the two agree to about 1e-13).  Each GPU result must have a
true relative residual <= 1e-8 and be within 1e-6 of the reference in

* the compliance f^T u (Eq. 1),
* ||u - u_ref||_2 / ||u_ref||_2, estimated from 8 seeded Gaussian projections of the whole
  vector and measured on 200 uniformly sampled DOFs,
* the largest error at the stored DOFs (sampled, loaded, largest |u|) relative to ||u_ref||_inf,
  within 1e-5: a pointwise error, which the displacement criterion (a relative error of the
  whole vector) does not bound; at a 1e-8 residual on the 1e9-contrast 2D design it is about
  1e-6 and moves with rounding-level changes of the hierarchy.

The largest 3D grid whose direct solve the oracle finishes within the test budget is
32x16x16 (28,611 DOFs, about 8 s); there the whole displacement vector is compared.
"""
import os
import sys

import numpy as np
import pytest

import workloads as W
from oracle import solve as osolve

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import refs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-6
MAXTOL = 1e-5  # pointwise error relative to ||u_ref||_inf (see above)
HYB3 = dict(pc="hybrid", n_geo_levels=3, max_coarse_dofs=1000, rtol=1e-8, max_iter=2000)


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def check(u, res, ref, G):
    assert res["status"] == 0 and res["rel_residual"] <= 1e-8, res
    acc = refs.accuracy(u, res["compliance"], ref, G)
    for k in ("rel_compliance_error", "rel_u_error_est", "rel_u_error_sampled"):
        assert acc[k] <= TOL, (k, acc)
    assert acc["max_abs_error_rel_inf"] <= MAXTOL, acc
    return acc


@pytest.fixture(scope="module")
def cant3d():
    p = W.cantilever_3d(192, 96, 96, seed=0)
    return p, refs.load("cantilever3d_192x96x96")[0], refs.projections(p.n)


@pytest.mark.parametrize("prec,smoother", [("tc", "chebyshev"), ("fp32", "chebyshev"),
                                           ("fp64", "chebyshev"), ("tc", "jacobi")])
def test_cantilever3d_full_vs_oracle(lib, ctx, cant3d, prec, smoother):
    p, ref, G = cant3d
    P = lib.Problem.from_workload(ctx, p)
    P.setup(prec=prec, smoother=smoother, cheb_degree=2, **HYB3)
    u, res = P.solve(p.f)
    check(u[0], res[0], ref, G)


@pytest.fixture(scope="module")
def batched():
    p = W.batched_3d()
    return p, refs.load("batched3d_128x64x64"), refs.projections(p.n)


@pytest.mark.parametrize("prec,smoother,conc,block", [("tc", "chebyshev", 4, 0),
                                                      ("fp32", "jacobi", 1, 0),
                                                      ("tc", "chebyshev", 1, 16)])
def test_batched_full_vs_oracle(lib, ctx, batched, prec, smoother, conc, block):
    """The 16 right-hand sides on concurrent solve slots, one at a time, and as one block solve
    (block_rhs = 16: every launch of the loop covers all 16)."""
    p, ref, G = batched
    P = lib.Problem.from_workload(ctx, p)
    P.setup(prec=prec, smoother=smoother, cheb_degree=2, concurrency=conc, block_rhs=block, **HYB3)
    u, res = P.solve(p.f)
    assert len(res) == 16
    for j in range(16):
        check(u[j], res[j], ref[j], G)


@pytest.mark.parametrize("pc", ["hybrid", "amg"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cantilever2d_full_vs_oracle(lib, ctx, pc, prec):
    """The algebraic hierarchies (SA-AMG from the fine level, and the hybrid).  A purely
    geometric hierarchy on these 0/1 members with 1e9 contrast stalls far above 1e-8 (the
    paper's motivation for AMG, Sec. 4.1); the bench reports it as not converged."""
    p = W.cantilever_2d(768, 384, seed=0)
    ref = refs.load("cantilever2d_768x384")[0]
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc=pc, prec=prec, smoother="chebyshev", cheb_degree=2, max_coarse_dofs=1500,
            n_geo_levels=2, rtol=1e-8, max_iter=2000)
    u, res = P.solve(p.f)
    check(u[0], res[0], ref, refs.projections(p.n))


def test_mbb_gmg4_fp64_jacobi_vs_oracle(lib, ctx):
    """The MBB beam as configured: FP64 GMG-PCG, 4 levels (12x4 coarse grid, 130 DOFs), one
    point-block Jacobi sweep."""
    p = W.mbb_beam(96, 32)
    ref = refs.load("mbb_96x32")[0]
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", prec="fp64", n_levels=4, smoother="jacobi", rtol=1e-8)
    assert P.level_info(3)["n_dofs"] == 130
    u, res = P.solve(p.f)
    check(u[0], res[0], ref, refs.projections(p.n))


@pytest.mark.parametrize("prec", ["tc", "fp32", "fp64"])
def test_cantilever3d_32x16x16_vs_direct(lib, ctx, prec):
    p = W.cantilever_3d(32, 16, 16, seed=0)
    ref = osolve.direct(p)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(prec=prec, smoother="chebyshev", cheb_degree=2, **HYB3)
    u, res = P.solve(p.f)
    assert res[0]["status"] == 0 and res[0]["rel_residual"] <= 1e-8
    d = u[0] - ref["u"][0]
    assert np.linalg.norm(d) <= TOL * np.linalg.norm(ref["u"][0])
    assert abs(res[0]["compliance"] - ref["compliance"][0]) <= TOL * abs(ref["compliance"][0])
