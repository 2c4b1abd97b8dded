"""GPU parity of the stability problem (Sec. 2.2; Algorithm 2): the stress stiffness operator
against the oracle's assembled K_sigma, and the generalized Davidson eigenvalues against dense
generalized eigenvalues (scipy) and the oracle's Davidson, on the same seeded inputs."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import fem, mg, solve as osolve, stability

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


@pytest.mark.parametrize("dim,grid", [(2, (7, 5, 1)), (2, (33, 17, 1)), (3, (5, 4, 3)),
                                      (3, (9, 6, 7))])
def test_stress_stiffness_apply(lib, ctx, dim, grid):
    """y = K_sigma(u) x: FP64, bound 1e-13 of the summed magnitudes |K_sigma| |x|."""
    p = W.random_problem(dim, *grid, seed=51, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    rng = np.random.default_rng(8)
    u = rng.standard_normal(p.n) * fem.free_mask(p.n, p.fixed)
    x = rng.standard_normal(p.n)
    Ks = stability.stress_stiffness(p, u)
    y = P.stress_stiffness_apply(u, x)
    scale = abs(Ks) @ np.abs(x)
    assert np.all(np.abs(y - Ks @ x) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_buckling_column_matches_dense(lib, ctx, prec):
    p = W.column_2d(8, 64)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=3, prec=prec, rtol=1e-12)
    u, res = P.solve(p.f)
    lam, Phi, it, st = P.buckling(u[0], n_eig=6, tol=1e-9, max_iter=2000, modes=True)
    assert st == 0
    A0 = mg.fine_operator(p)
    uref = osolve.direct(p)["u"][0]
    Ks = stability.stress_stiffness(p, uref)
    ref = sla.eigh(Ks.toarray(), A0.toarray(), eigvals_only=True)[::-1][:6]
    assert np.allclose(lam, ref, rtol=1e-7)
    assert np.allclose(Phi @ (A0 @ Phi.T), np.eye(6), atol=1e-7)
    # each mode satisfies the eigen-equation
    for i in range(6):
        rr = Ks @ Phi[i] - lam[i] * (A0 @ Phi[i])
        assert np.linalg.norm(rr) <= 1e-6 * abs(lam[i]) * np.linalg.norm(A0 @ Phi[i])
    # Euler's load of a fixed-free column within 5 %
    pcr = np.pi ** 2 * 8 ** 3 / 12.0 / (4.0 * 64 ** 2)
    assert 1.0 / lam[0] == pytest.approx(pcr, rel=0.05)


def test_buckling_3d_and_random_column_vs_oracle(lib, ctx):
    p = W.column_2d(24, 96, seed=3)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="hybrid", n_geo_levels=2, max_coarse_dofs=300, prec="fp32", rtol=1e-12)
    u, _ = P.solve(p.f)
    lam, _, it, st = P.buckling(u[0], n_eig=6, tol=1e-8)
    assert st == 0
    A0 = mg.fine_operator(p)
    Ks = stability.stress_stiffness(p, osolve.direct(p)["u"][0])
    H = osolve.build(p, pc="hybrid", n_geo=2, cap=300)
    th, _, oit, _ = stability.davidson(Ks, A0, M=lambda v: mg.vcycle(H, v), n_eig=6, tol=1e-8)
    assert np.allclose(lam, th, rtol=1e-6)
    # a 3D clamped block under its own face load
    q = W.random_problem(3, 6, 5, 4, seed=52, contrast="minmax")
    Q = lib.Problem.from_workload(ctx, q)
    Q.setup(pc="gmg", n_levels=2, prec="fp64", rtol=1e-12)
    uq, _ = Q.solve(q.f)
    lq, _, _, stq = Q.buckling(uq[0], n_eig=4, tol=1e-9)
    assert stq == 0
    Kq = stability.stress_stiffness(q, osolve.direct(q)["u"][0])
    refq = sla.eigh(Kq.toarray(), mg.fine_operator(q).toarray(), eigvals_only=True)[::-1][:4]
    assert np.allclose(lq, refq, rtol=1e-7)


def test_buckling_invalid(lib, ctx):
    p = W.column_2d(4, 8)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=2)
    u, _ = P.solve(p.f)
    for kw in (dict(n_eig=0), dict(n_eig=6, j_min=6), dict(j_min=10, j_max=10),
               dict(j_max=65), dict(tol=0.0)):
        with pytest.raises(lib.TomgError):
            P.buckling(u[0], **kw)


def _dense_modes(p, k):
    """The k largest eigenpairs (K-normalised) of the oracle's dense generalized problem, the
    direct displacements, the adjoint solutions and the masked operator."""
    u = osolve.direct(p)["u"][0]
    A0 = mg.fine_operator(p)
    lam, Z = sla.eigh(stability.stress_stiffness(p, u).toarray(), A0.toarray())
    lam, Z = lam[::-1][:k], Z[:, ::-1][:, :k].T.copy()
    V = np.array([np.linalg.solve(A0.toarray(), stability.adjoint_rhs(p, z)) for z in Z])
    return u, lam, Z, V, A0


@pytest.mark.parametrize("dim,grid", [(2, (7, 5, 1)), (2, (33, 17, 1)), (3, (5, 4, 3)),
                                      (3, (9, 6, 7))])
def test_adjoint_rhs(lib, ctx, dim, grid):
    """g_k = Phi_k^T (dK_sigma/du) Phi_k for three random vectors (FP64; rounding of sums of
    at most 2^d element terms), host and device paths."""
    p = W.random_problem(dim, *grid, seed=53, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    Phi = np.random.default_rng(9).standard_normal((3, p.n))
    g = P.buckling_adjoint_rhs(Phi)
    for k in range(3):
        ref = stability.adjoint_rhs(p, Phi[k])
        assert np.abs(g[k] - ref).max() <= 1e-12 * np.abs(ref).max()
    import torch
    gd = P.buckling_adjoint_rhs(torch.from_numpy(Phi).cuda())
    assert np.array_equal(gd.cpu().numpy(), g)


@pytest.mark.parametrize("dim,grid", [(2, (6, 16, 1)), (3, (3, 3, 5))])
def test_buckling_sensitivity_kernel(lib, ctx, dim, grid):
    """dlambda_k/drho_e, dF/drho_e and F on the oracle's exact u, modes and adjoint solutions
    (densities on both sides of the E_sigma cutoff): FP64, 1e-11 of the largest entry."""
    p = W.random_problem(dim, *grid, seed=54, contrast="minmax")
    assert np.any(p.rho < 0.1)
    u, lam, Z, V, _ = _dense_modes(p, 4)
    P = lib.Problem.from_workload(ctx, p)
    dl, dF, F = P.buckling_sensitivity(u, lam, Z, V, pnorm=8)
    ref = np.array([stability.eigenvalue_sensitivity(p, u, lam[k], Z[k], V[k]) for k in range(4)])
    assert np.abs(dl - ref).max() <= 1e-11 * np.abs(ref).max()
    assert F == pytest.approx(stability.pnorm(lam), rel=1e-14)
    rF = stability.pnorm_sensitivity(lam, ref)
    assert np.abs(dF - rF).max() <= 1e-11 * np.abs(rF).max()
    import torch
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    dld, dFd, Fd = P.buckling_sensitivity(cu(u), lam, cu(Z), cu(V), pnorm=8)
    assert np.array_equal(dld.cpu().numpy(), dl) and np.array_equal(dFd.cpu().numpy(), dF)
    assert Fd == F


def test_buckling_sensitivity_chain(lib, ctx):
    """The whole chain on the GPU (solve, Davidson, adjoint right-hand sides, adjoint solves on
    concurrent slots, sensitivities, filter transpose) against the oracle's dense chain on a
    seeded column.  The GPU modes carry the Davidson tolerance, so the bound is 1e-5 of the
    largest sensitivity."""
    p = W.column_2d(12, 40, seed=5, sigma=3.0)
    u, lam, Z, V, _ = _dense_modes(p, 7)
    assert np.all(np.diff(lam) < -1e-3 * lam[0])
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=3, prec="fp32", rtol=1e-10, concurrency=6)
    ug, r0 = P.solve(p.f)
    assert r0[0]["status"] == 0, r0
    lg, Phi, _, st = P.buckling(ug[0], n_eig=6, tol=1e-10, max_iter=3000, modes=True)
    assert st == 0 and np.allclose(lg, lam[:6], rtol=1e-9)
    g = P.buckling_adjoint_rhs(Phi)
    vg, res = P.solve(g)
    assert all(r["status"] == 0 for r in res), res
    dl, dF, F = P.buckling_sensitivity(ug[0], lg, Phi, vg, pnorm=8)
    ref = np.array([stability.eigenvalue_sensitivity(p, u, lam[k], Z[k], V[k]) for k in range(6)])
    assert np.abs(dl - ref).max() <= 1e-5 * np.abs(ref).max()
    rF = stability.pnorm_sensitivity(lam[:6], ref)
    assert np.abs(dF - rF).max() <= 1e-5 * np.abs(rF).max()
    from oracle import design
    S = design.filter_matrix(2, p.nx, p.ny, 1, 1.5)
    da = P.density_filter(dF, radius=1.5, transpose=True)
    assert np.abs(da - S.T @ rF).max() <= 1e-5 * np.abs(S.T @ rF).max()


def test_buckling_sensitivity_invalid(lib, ctx):
    p = W.column_2d(4, 8)
    P = lib.Problem.from_workload(ctx, p)
    z = np.zeros((2, p.n))
    for nm in (0, 17):
        with pytest.raises(lib.TomgError):
            P.buckling_adjoint_rhs(np.zeros((nm, p.n)) if nm else np.zeros((1, p.n))[:0])
    for lam, pn in (([1.0, 2.0], 0.5), ([-1.0, -2.0], 3.0), ([0.0, 0.0], 8.0)):
        with pytest.raises(lib.TomgError):
            P.buckling_sensitivity(np.zeros(p.n), lam, z, z, pnorm=pn)
