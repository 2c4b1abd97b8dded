"""Pins for oracle.stability: the stress stiffness matrix and the generalized Davidson solver."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import fem, mg, solve, stability


def _int01(c, d):
    """Exact integral over [0, 1] of (c0 + c1 x)(d0 + d1 x)."""
    return c[0] * d[0] + Fraction(c[0] * d[1] + c[1] * d[0], 2) + Fraction(c[1] * d[1], 3)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_products_exact(dim):
    """L_ij[a, b] against exact rational integration of the factorised multilinear functions."""
    L = stability.gradient_products(dim)
    nn = 1 << dim
    for i in range(dim):
        for j in range(dim):
            for a in range(nn):
                for b in range(nn):
                    tot = Fraction(1)
                    for m in range(dim):
                        def factor(node, deriv_axis):
                            bit = (node >> m) & 1
                            if m == deriv_axis:
                                return (Fraction(1 if bit else -1), Fraction(0))
                            return (Fraction(0), Fraction(1)) if bit else (Fraction(1), Fraction(-1))
                        tot *= _int01(factor(a, i), factor(b, j))
                    assert L[i, j, a, b] == pytest.approx(float(tot), abs=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_strain_stresses(dim):
    """A linear displacement field has the same stress in every element: E_sigma D0 eps."""
    p = W.random_problem(dim, 4, 3, 2, seed=6, contrast="minmax")
    c = fem.node_coords(dim, p.nx, p.ny, p.nz)
    G = np.random.default_rng(1).standard_normal((dim, dim))
    u = (c @ G.T).ravel()  # u(x) = G x
    eps_t = 0.5 * (G + G.T)
    if dim == 2:
        eps = np.array([eps_t[0, 0], eps_t[1, 1], 2 * eps_t[0, 1]])
    else:
        eps = np.array([eps_t[0, 0], eps_t[1, 1], eps_t[2, 2], 2 * eps_t[1, 2], 2 * eps_t[0, 2],
                        2 * eps_t[0, 1]])
    sv = fem.constitutive(dim, 1.0, p.nu) @ eps
    S = stability.element_stresses(p, u)
    Es = stability.stress_interp(p.rho, p.E0, p.penal)
    assert np.all(Es[p.rho < 0.1] == 0.0)
    for e in range(S.shape[0]):
        ref = Es[e] * sv
        got = [S[e, 0, 0], S[e, 1, 1], S[e, 0, 1]] if dim == 2 else \
            [S[e, 0, 0], S[e, 1, 1], S[e, 2, 2], S[e, 1, 2], S[e, 0, 2], S[e, 0, 1]]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_stress_stiffness_symmetric_translation_free(dim):
    p = W.random_problem(dim, 5, 3, 3, seed=7, contrast="minmax")
    u = np.random.default_rng(2).standard_normal(p.n) * fem.free_mask(p.n, p.fixed)
    Ks = stability.stress_stiffness(p, u)
    assert abs(Ks - Ks.T).max() <= 1e-14 * abs(Ks).max()
    free = fem.free_mask(p.n, p.fixed).astype(bool)
    # unmasked K_G annihilates rigid translations: check through an unmasked problem
    q = W.Problem(p.name, dim, p.nx, p.ny, p.nz, p.rho, np.array([], dtype=np.int64), p.f,
                  E0=p.E0, Emin=p.Emin, penal=p.penal, nu=p.nu)
    Kq = stability.stress_stiffness(q, u)
    for c in range(dim):
        t = np.zeros(p.n)
        t[c::dim] = 1.0
        assert np.abs(Kq @ t).max() <= 1e-12 * abs(Kq).max()
    assert np.all(Ks.toarray()[~free] == 0.0)


def _column(nx=4, ny=16):
    """A column clamped at y = 0 with a downward unit load spread over its top edge."""
    return W.column_2d(nx, ny)


@pytest.mark.parametrize("precond", ["identity", "direct", "vcycle"])
def test_davidson_matches_dense(precond):
    p = _column()
    A0 = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * p.f[0]
    u = solve.direct(p)["u"][0]
    Ks = stability.stress_stiffness(p, u)
    lam = sla.eigh(Ks.toarray(), A0.toarray(), eigvals_only=True)[::-1][:6]
    assert lam[0] > 0
    if precond == "identity":
        M = None
    elif precond == "direct":
        import scipy.sparse.linalg as spla
        lu = spla.splu(A0.tocsc())
        M = lu.solve
    else:
        H = solve.build(p, pc="gmg", n_levels=3)
        M = lambda v: mg.vcycle(H, v)  # noqa: E731
    th, Phi, it, res = stability.davidson(Ks, A0, M=M, n_eig=6, tol=1e-9, max_iter=2000)
    assert np.allclose(th, lam, rtol=1e-8)
    assert np.allclose(Phi.T @ (A0 @ Phi), np.eye(6), atol=1e-8)
    if precond == "direct":
        assert it < 200


def test_column_buckling_load_matches_euler():
    """A slender solid fixed-free column under an end load buckles at Euler's
    P_cr = pi^2 E I / (4 L^2) (I = width^3 / 12 per unit thickness, E = 1): 1 / lambda_max must
    come within a few per cent (the FE column is not perfectly slender; shear and the discrete
    bending stiffness of one element row account for the rest)."""
    nx, ny = 8, 64
    p = W.column_2d(nx, ny)
    A0 = mg.fine_operator(p)
    u = solve.direct(p)["u"][0]
    Ks = stability.stress_stiffness(p, u)
    H = solve.build(p, pc="gmg", n_levels=3)
    th, _, _, _ = stability.davidson(Ks, A0, M=lambda v: mg.vcycle(H, v), n_eig=2, tol=1e-8)
    pcr = np.pi ** 2 * nx ** 3 / 12.0 / (4.0 * ny ** 2)
    assert 1.0 / th[0] == pytest.approx(pcr, rel=0.05)


def _with_rho(p, rho):
    return W.Problem(p.name, p.dim, p.nx, p.ny, p.nz, np.asarray(rho, dtype=np.float64), p.fixed,
                     p.f, E0=p.E0, Emin=p.Emin, penal=p.penal, nu=p.nu)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_rhs_brute_force(dim):
    """g_i = Phi^T K_sigma(e_i) Phi for every free DOF i (K_sigma is linear in u), 0 at fixed
    DOFs; the density spans the E_sigma cutoff so elements with E_sigma = 0 are included."""
    p = W.random_problem(dim, 4, 3, 2, seed=8, contrast="minmax")
    assert np.any(p.rho < 0.1) and np.any(p.rho >= 0.1)
    free = fem.free_mask(p.n, p.fixed).astype(bool)
    phi = np.random.default_rng(3).standard_normal(p.n) * free
    g = stability.adjoint_rhs(p, phi)
    ref = np.zeros(p.n)
    for i in np.flatnonzero(free):
        e = np.zeros(p.n)
        e[i] = 1.0
        ref[i] = phi @ (stability.stress_stiffness(p, e) @ phi)
    assert np.all(g[~free] == 0.0)
    assert np.allclose(g, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def _dense_buckling(p):
    u = solve.direct(p)["u"][0]
    Ks = stability.stress_stiffness(p, u).toarray()
    K = mg.fine_operator(p).toarray()
    lam, Z = sla.eigh(Ks, K)
    return lam[::-1], Z[:, ::-1], u, K


def _sensitivity_case(dim):
    if dim == 2:
        p = W.column_2d(3, 8)
    else:
        p = W.random_problem(3, 2, 2, 3, seed=4, contrast="minmax")
    rho = np.random.default_rng(11).uniform(0.3, 1.0, p.nel)  # clear of the 0.1 cutoff
    return _with_rho(p, rho)


@pytest.mark.parametrize("dim", [2, 3])
def test_eigenvalue_sensitivity_finite_differences(dim):
    """dlambda/drho_e of the three largest (simple) eigenvalues against central differences of
    dense generalized eigenvalues, u re-solved at every perturbed density.  The adjoint term is
    large here: flipping its sign (the paper's printed +) misses by far more than the bound."""
    p = _sensitivity_case(dim)
    lam, Z, u, K = _dense_buckling(p)
    assert np.all(np.diff(lam[:4]) < -1e-3 * abs(lam[0]))  # simple eigenvalues
    h = 1e-5
    for k in range(3):
        phi = Z[:, k]
        v = np.linalg.solve(K, stability.adjoint_rhs(p, phi))
        d = stability.eigenvalue_sensitivity(p, u, lam[k], phi, v)
        fd = np.zeros(p.nel)
        for e in range(p.nel):
            r1, r2 = p.rho.copy(), p.rho.copy()
            r1[e] += h
            r2[e] -= h
            fd[e] = (_dense_buckling(_with_rho(p, r1))[0][k] -
                     _dense_buckling(_with_rho(p, r2))[0][k]) / (2 * h)
        scale = np.abs(fd).max()
        assert np.abs(d - fd).max() <= 1e-6 * scale
        flipped = stability.eigenvalue_sensitivity(p, u, lam[k], phi, -v)
        assert np.abs(flipped - fd).max() > 1e-2 * scale


def test_pnorm_closed_forms():
    assert stability.pnorm([3.0]) == pytest.approx(3.0, rel=1e-15)
    assert stability.pnorm([2.0] * 6) == pytest.approx(2.0 * 6 ** 0.125, rel=1e-15)
    assert stability.pnorm([3.0, 4.0], p=2) == pytest.approx(5.0, rel=1e-15)


def test_pnorm_sensitivity_finite_differences():
    """dF/drho of the p = 8 norm of the three largest eigenvalues against central differences."""
    p = _sensitivity_case(2)
    lam, Z, u, K = _dense_buckling(p)
    n = 3
    dl = []
    for k in range(n):
        v = np.linalg.solve(K, stability.adjoint_rhs(p, Z[:, k]))
        dl.append(stability.eigenvalue_sensitivity(p, u, lam[k], Z[:, k], v))
    dF = stability.pnorm_sensitivity(lam[:n], np.array(dl))
    h = 1e-5
    fd = np.zeros(p.nel)
    for e in range(p.nel):
        r1, r2 = p.rho.copy(), p.rho.copy()
        r1[e] += h
        r2[e] -= h
        fd[e] = (stability.pnorm(_dense_buckling(_with_rho(p, r1))[0][:n]) -
                 stability.pnorm(_dense_buckling(_with_rho(p, r2))[0][:n])) / (2 * h)
    assert np.abs(dF - fd).max() <= 1e-6 * np.abs(fd).max()
