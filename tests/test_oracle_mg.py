"""Pins for oracle.mg (V-cycle, hierarchies) and oracle.krylov (PCG / FCG)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, gmg, krylov, mg, solve


def _hier(kind, p, **kw):
    if kind == "gmg":
        return solve.build(p, pc="gmg", n_levels=3, **kw)
    if kind == "amg":
        return solve.build(p, pc="amg", cap=60, **kw)
    return solve.build(p, pc="hybrid", n_geo=2, cap=60, **kw)


@pytest.mark.parametrize("kind", ["gmg", "amg", "hybrid"])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_vcycle_symmetric_and_contracting(kind, smoother):
    p = W.random_problem(2, 16, 8, seed=8, contrast="minmax")
    H = _hier(kind, p, smoother=smoother)
    A = H.A[0]
    n = A.shape[0]
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    Mx, My = mg.vcycle(H, x), mg.vcycle(H, y)
    assert abs(x @ My - y @ Mx) <= 1e-10 * abs(x @ My)
    # M^-1 SPD on random vectors
    assert x @ Mx > 0 and y @ My > 0
    # error propagation I - M^-1 A contracts in the A-norm
    e = rng.standard_normal(n)
    e2 = e - mg.vcycle(H, A @ e)
    assert np.sqrt(e2 @ (A @ e2)) < np.sqrt(e @ (A @ e))


def test_one_level_is_exact():
    p = W.random_problem(2, 6, 4, seed=9, contrast="minmax")
    H = solve.build(p, pc="gmg", n_levels=1)
    b = np.random.default_rng(1).standard_normal(p.n)
    assert np.allclose(H.A[0] @ mg.vcycle(H, b), b, atol=1e-9 * np.abs(b).max())


def test_vcycle_matches_algorithm1_by_hand():
    """Two-level cycle written out with dense matrices: pre-smooth, restrict, exact coarse
    solve, prolong, post-smooth."""
    p = W.random_problem(2, 6, 4, seed=10, contrast="minmax")
    H = solve.build(p, pc="gmg", n_levels=2)
    A, P = H.A[0].toarray(), H.P[0].toarray()
    Ac = P.T @ A @ P
    n = A.shape[0]
    Db = np.zeros_like(A)
    for i in range(0, n, 2):
        Db[i:i + 2, i:i + 2] = A[i:i + 2, i:i + 2]
    Dinv = np.linalg.inv(Db)
    b = np.random.default_rng(2).standard_normal(n)
    x = 0.5 * Dinv @ b
    x = x + P @ np.linalg.solve(Ac, P.T @ (b - A @ x))
    x = x + 0.5 * Dinv @ (b - A @ x)
    assert np.allclose(mg.vcycle(H, b), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_gmg_iterations_bounded_under_refinement():
    """Uniform density: GMG-PCG iteration counts stay roughly constant as the grid is refined
    (Sec. 3.2: multigrid convergence independent of the grid size)."""
    its = []
    for s in (1, 2, 4):
        p = W.mbb_beam(24 * s, 8 * s)
        r = solve.solve(p, pc="gmg", n_levels=2 + s // 2 + (s == 4))
        its.append(int(r["iterations"][0]))
    assert max(its) <= 2.0 * min(its) + 4


@pytest.mark.parametrize("pc,kw", [("gmg", dict(n_levels=4)), ("amg", dict(cap=130)),
                                  ("hybrid", dict(n_geo=2, cap=130))])
def test_pcg_matches_direct_mbb(pc, kw):
    p = W.mbb_beam(96, 32)
    ref = solve.direct(p)
    r = solve.solve(p, pc=pc, rtol=1e-10, **kw)
    assert r["rel_residual"][0] <= 1e-10 * 1.01
    err = np.linalg.norm(r["u"] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-8
    assert r["compliance"][0] == pytest.approx(ref["compliance"][0], rel=1e-9)


def test_pcg_exact_in_n_steps_and_zero_rhs():
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((12, 12))
    A = Q @ Q.T + 12 * np.eye(12)
    b = rng.standard_normal(12)
    x, it, _ = krylov.pcg(A, b, rtol=1e-13, max_iter=100)
    assert it <= 12 + 2
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    x0, it0, _ = krylov.pcg(A, np.zeros(12))
    assert it0 == 0 and np.all(x0 == 0)


def test_fcg_equals_pcg_for_fixed_spd_preconditioner():
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((30, 30))
    A = Q @ Q.T + np.eye(30)
    Minv = np.diag(1.0 / np.diag(A))
    b = rng.standard_normal(30)
    x1, i1, h1 = krylov.pcg(A, b, M=lambda r: Minv @ r, rtol=1e-10)
    x2, i2, h2 = krylov.pcg(A, b, M=lambda r: Minv @ r, rtol=1e-10, flexible=True)
    assert abs(i1 - i2) <= 2
    assert np.allclose(h1[:20], h2[:20], rtol=1e-8)  # before the n-step finite-precision tail
    assert np.allclose(x1, x2, rtol=1e-8)


def test_warm_start_from_solution_takes_zero_iterations():
    p = W.mbb_beam(24, 8)
    ref = solve.direct(p)
    r = solve.solve(p, pc="gmg", n_levels=2, x0=ref["u"])
    assert r["iterations"][0] == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_through_pcg(dim):
    p = W.patch_tension(dim, 8, 4, 4, sigma=1.0, E=1.0)
    r = solve.solve(p, pc="gmg", n_levels=2, rtol=1e-12)
    X = fem.node_coords(dim, p.nx, p.ny, p.nz)
    ex = np.zeros_like(X)
    ex[:, 0] = X[:, 0]
    for c in range(1, dim):
        ex[:, c] = -0.3 * X[:, c]
    assert np.allclose(r["u"][0].reshape(-1, dim), ex, atol=1e-9)


def _small_spd_with_blocks():
    p = W.random_problem(2, 6, 4, seed=17, contrast="minmax")
    A = mg.fine_operator(p)
    from oracle import amg
    Dinv = amg.block_diag_inv(A, 2)
    return A, Dinv


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_chebyshev_error_is_scaled_chebyshev_polynomial(m):
    """Error propagation of m Chebyshev steps: e_m = p_m(D^-1 A) e_0 with
    p_m(t) = T_m((theta - t) / delta) / T_m(theta / delta) (the defining property of Chebyshev
    acceleration on [a, b]).  On every generalized eigenvector A v = lam D v the smoother must
    scale v by p_m(lam); T_m is evaluated by numpy's Chebyshev series routine.  A dropped term,
    a wrong sign or an index slip in the recurrence changes p_m."""
    import scipy.linalg as sla
    from numpy.polynomial import chebyshev as C
    A, Dinv = _small_spd_with_blocks()
    Ad = A.toarray()
    n = Ad.shape[0]
    D = np.zeros_like(Ad)
    for i in range(0, n, 2):
        D[i:i + 2, i:i + 2] = np.linalg.inv(Dinv[i // 2])
    lam, V = sla.eigh(Ad, D)
    a, b = 0.1 * lam.max(), 1.1 * lam.max()
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    Tm = np.zeros(m + 1)
    Tm[m] = 1.0
    p = C.chebval((theta - lam) / delta, Tm) / C.chebval(theta / delta, Tm)
    for i in range(0, n, max(1, n // 12)):
        v = V[:, i]
        out = mg.chebyshev_smooth(A, Dinv, v.copy(), np.zeros(n), a, b, m)
        assert np.allclose(out, p[i] * v, rtol=0, atol=1e-11 * np.abs(v).max()), (m, i)
    # on [a, b] the polynomial is bounded by 1 / T_m(theta / delta)
    inside = (lam >= a) & (lam <= b)
    assert np.all(np.abs(p[inside]) <= 1.0 / C.chebval(theta / delta, Tm) + 1e-12)


def test_chebyshev_degree_one_is_weighted_jacobi():
    A, Dinv = _small_spd_with_blocks()
    from oracle import amg
    rng = np.random.default_rng(3)
    x, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    lo, hi = 0.3, 3.7  # theta = 2: weight 1/2
    ref = x + 0.5 * amg.apply_block_diag(Dinv, b - A @ x)
    assert np.allclose(mg.chebyshev_smooth(A, Dinv, x, b, lo, hi, 1), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("case", ["mbb", "rand"])
def test_chebyshev_vcycle_cuts_iterations(case):
    """A degree-2 Chebyshev smoother is a stronger smoother than one Jacobi sweep: PCG needs
    fewer iterations (18 -> 10 on the MBB beam, 19 -> 11 on the random design)."""
    p = W.mbb_beam(96, 32) if case == "mbb" else W.random_problem(2, 64, 32, seed=5,
                                                                   contrast="minmax")
    rj = solve.solve(p, pc="gmg", n_levels=4)
    rc = solve.solve(p, pc="gmg", n_levels=4, smoother="chebyshev", cheb_degree=2)
    assert rc["rel_residual"][0] <= 1e-8 and rj["rel_residual"][0] <= 1e-8
    assert rc["iterations"][0] < rj["iterations"][0]


def _small_system(seed=19):
    p = W.random_problem(2, 5, 3, seed=seed, contrast="minmax")
    A = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * np.random.default_rng(seed).standard_normal(p.n)
    return p, A, b


@pytest.mark.parametrize("k", [1, 3, 6, 10])
def test_fgmres_minimal_residual_over_krylov_space(k):
    """After k Arnoldi steps of one cycle, FGMRES with a fixed preconditioner M minimises
    ||b - A x|| over x in span{M v_0, ..., M v_{k-1}} = M K_k(A M, b): brute force builds that
    space from powers of A M applied to b and solves the least-squares problem with lstsq."""
    p, A, b = _small_system()
    Ad = A.toarray()
    Dinv = np.diag(1.0 / np.diag(Ad))
    Mfun = lambda v: Dinv @ v  # noqa: E731
    x, it, hist = krylov.fgmres(A, b, M=Mfun, rtol=0.0, max_iter=k, restart=50)
    assert it == k
    Kb = [b / np.linalg.norm(b)]
    for _ in range(k - 1):
        v = Ad @ (Dinv @ Kb[-1])
        Kb.append(v / np.linalg.norm(v))
    Y = Dinv @ np.stack(Kb, axis=1)
    c, *_ = np.linalg.lstsq(Ad @ Y, b, rcond=None)
    best = np.linalg.norm(b - Ad @ (Y @ c))
    assert np.linalg.norm(b - Ad @ x) == pytest.approx(best, rel=1e-7, abs=1e-12 * np.linalg.norm(b))
    # the Givens estimate of the last step is the true residual of that cycle's iterate
    assert hist[-1] * np.linalg.norm(b) == pytest.approx(np.linalg.norm(b - Ad @ x), rel=1e-6)


def test_fgmres_finite_termination_and_monotone():
    """Without restarts GMRES ends in at most n steps (exactly so in exact arithmetic; on a
    well-conditioned operator -- uniform density -- also in FP64)."""
    p = W.mbb_beam(6, 3)
    A = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * np.random.default_rng(20).standard_normal(p.n)
    n = A.shape[0]
    x, it, hist = krylov.fgmres(A, b, rtol=1e-12, max_iter=2 * n, restart=n + 1)
    assert it <= n
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    steps = hist[1:-1]  # the Givens estimates of the one cycle (the last entry: true residual)
    assert all(steps[i + 1] <= steps[i] * (1 + 1e-12) for i in range(len(steps) - 1))


@pytest.mark.parametrize("restart", [5, 30])
def test_fgmres_vcycle_matches_direct(restart):
    p = W.mbb_beam(48, 16)
    r = solve.solve(p, pc="gmg", n_levels=3, krylov_method="fgmres", restart=restart)
    ref = solve.direct(p)
    assert r["rel_residual"][0] <= 1e-8
    assert np.linalg.norm(r["u"] - ref["u"]) <= 1e-6 * np.linalg.norm(ref["u"])


@pytest.mark.parametrize("m", [1, 2, 4])
@pytest.mark.parametrize("warm", [False, True])
def test_gmres_smoother_minimises_over_power_basis(m, warm):
    """m GMRES smoothing steps from x0 give the minimiser of ||b - A x|| over
    x0 + D^-1 K_m(A D^-1, r0): brute force builds the space from powers of A D^-1 applied to r0
    (no Arnoldi) and solves the least-squares problem with lstsq; the minimiser is unique."""
    p = W.random_problem(2, 6, 4, 1, seed=21, contrast="minmax")
    A = mg.fine_operator(p)
    Ad = A.toarray()
    H = solve.build(p, pc="gmg", n_levels=2)
    Dinv = H.Dinv[0]
    rng = np.random.default_rng(22)
    b = rng.standard_normal(p.n)
    x0 = rng.standard_normal(p.n) if warm else np.zeros(p.n)
    x = mg.gmres_smooth(A, Dinv, x0, b, m)
    from oracle import amg
    r0 = b - Ad @ x0
    Kb = [r0 / np.linalg.norm(r0)]
    for _ in range(m - 1):
        v = Ad @ amg.apply_block_diag(Dinv, Kb[-1])
        Kb.append(v / np.linalg.norm(v))
    Y = np.stack([amg.apply_block_diag(Dinv, k) for k in Kb], axis=1)
    c, *_ = np.linalg.lstsq(Ad @ Y, r0, rcond=None)
    ref = x0 + Y @ c
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
    # more steps never raise the residual
    if m > 1:
        xm = mg.gmres_smooth(A, Dinv, x0, b, m - 1)
        assert np.linalg.norm(b - Ad @ x) <= np.linalg.norm(b - Ad @ xm) * (1 + 1e-12)


def test_gmres_smoother_finite_termination_and_breakdowns():
    """m = n steps solve the system (uniform density, well conditioned); b = 0 from x0 = 0
    returns 0; with A block diagonal the first step already solves exactly (h_21 = 0 is an
    exact breakdown: D^-1 r0 is the solution) and later steps are not taken."""
    p = W.mbb_beam(3, 2)
    A = mg.fine_operator(p)
    H = solve.build(p, pc="gmg", n_levels=2)
    b = fem.free_mask(p.n, p.fixed) * np.random.default_rng(23).standard_normal(p.n)
    x = mg.gmres_smooth(A, H.Dinv[0], np.zeros(p.n), b, p.n)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    assert np.all(mg.gmres_smooth(A, H.Dinv[0], np.zeros(p.n), np.zeros(p.n), 3) == 0.0)
    # powers of two and a unit-norm v_1 keep every step exact, so h_21 is exactly 0
    d = 2.0 ** np.arange(8)
    Dinv = np.stack([np.diag(1.0 / d[2 * k:2 * k + 2]) for k in range(4)])
    bb = np.array([1.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 1.0])
    xd = mg.gmres_smooth(sp.diags(d).tocsr(), Dinv, np.zeros(8), bb, 3)
    assert np.array_equal(xd, bb / d)


@pytest.mark.parametrize("pc,kw", [("gmg", dict(n_levels=3)), ("hybrid", dict(n_geo=2, cap=80))])
def test_gmres_smoother_vcycle_solves(pc, kw):
    """Flexible CG and FGMRES with the GMRES-smoothed cycle reach the direct solution, in fewer
    iterations than with the Jacobi smoother (Sec. 4.1: the GMRES smoother needs the fewest)."""
    p = W.mbb_beam(48, 16)
    ref = solve.direct(p)
    rj = solve.solve(p, pc=pc, flexible=True, **kw)
    for method in ("cg", "fgmres"):
        r = solve.solve(p, pc=pc, smoother="gmres", krylov_method=method, **kw)
        assert r["rel_residual"][0] <= 1e-8
        assert np.linalg.norm(r["u"] - ref["u"]) <= 1e-6 * np.linalg.norm(ref["u"])
        assert r["iterations"][0] < rj["iterations"][0]
