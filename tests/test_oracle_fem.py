"""Pins for oracle.fem: element stiffness, assembly, boundary conditions, direct solve."""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import fem


# ---------- exact rational element stiffness, by symbolic polynomial integration ----------

def _pmul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return out


def _pint(p):
    s = Fraction(0)
    for e, c in p.items():
        t = Fraction(c)
        for k in e:
            t /= (k + 1)
        s += t
    return s


def _dshape(dim, a, k):
    """dN_a/dx_k as a polynomial {exponents: coefficient} on [0,1]^dim."""
    poly = {tuple([0] * dim): Fraction(1 if (a >> k) & 1 else -1)}
    for m in range(dim):
        if m == k:
            continue
        one = [0] * dim
        lin = [0] * dim
        lin[m] = 1
        if (a >> m) & 1:
            f = {tuple(lin): Fraction(1)}
        else:
            f = {tuple(one): Fraction(1), tuple(lin): Fraction(-1)}
        poly = _pmul(poly, f)
    return poly


def exact_ke(dim, nu):
    nu = Fraction(nu)
    if dim == 2:
        c = 1 / (1 - nu * nu)
        D = [[c, c * nu, 0], [c * nu, c, 0], [0, 0, c * (1 - nu) / 2]]
    else:
        lam = nu / ((1 + nu) * (1 - 2 * nu))
        mu = 1 / (2 * (1 + nu))
        D = [[0] * 6 for _ in range(6)]
        for i in range(3):
            for j in range(3):
                D[i][j] = lam + (2 * mu if i == j else 0)
        for i in range(3, 6):
            D[i][i] = mu
    nn = 1 << dim
    # strain rows as lists of (node, comp, derivative axis)
    if dim == 2:
        rows = [[(0, 0)], [(1, 1)], [(0, 1), (1, 0)]]  # (comp, axis): exx=du/dx, eyy, gxy
    else:
        rows = [[(0, 0)], [(1, 1)], [(2, 2)], [(1, 2), (2, 1)], [(0, 2), (2, 0)], [(0, 1), (1, 0)]]
    nd = dim * nn
    # B as polynomials: B[s][dof]
    B = [[{} for _ in range(nd)] for _ in range(len(rows))]
    for s, terms in enumerate(rows):
        for a in range(nn):
            for comp, ax in terms:
                B[s][dim * a + comp] = _dshape(dim, a, ax)
    Ke = np.zeros((nd, nd))
    for i in range(nd):
        for j in range(i, nd):
            tot = Fraction(0)
            for s in range(len(rows)):
                if not B[s][i]:
                    continue
                for t in range(len(rows)):
                    if D[s][t] == 0 or not B[t][j]:
                        continue
                    tot += D[s][t] * _pint(_pmul(B[s][i], B[t][j]))
            Ke[i, j] = Ke[j, i] = float(tot)
    return Ke


@pytest.mark.parametrize("dim", [2, 3])
def test_ke_matches_exact_integration(dim):
    Ke = fem.element_stiffness(dim, 0.3)
    Kx = exact_ke(dim, Fraction(3, 10))
    assert np.max(np.abs(Ke - Kx)) <= 1e-15 * np.max(np.abs(Kx)) * 10


def test_ke_quad4_textbook():
    """Closed-form bilinear plane-stress element matrix (e.g. Andreassen et al. 2011, top88):
    k = [1/2-nu/6, 1/8+nu/8, -1/4-nu/12, -1/8+3nu/8, -1/4+nu/12, -1/8-nu/8, nu/6, 1/8-3nu/8]
    with nodes ordered counter-clockwise from the lower-left corner."""
    nu = 0.3
    k = [0.5 - nu / 6, 0.125 + nu / 8, -0.25 - nu / 12, -0.125 + 3 * nu / 8,
         -0.25 + nu / 12, -0.125 - nu / 8, nu / 6, 0.125 - 3 * nu / 8]
    k1, k2, k3, k4, k5, k6, k7, k8 = k
    KE = 1 / (1 - nu ** 2) * np.array([
        [k1, k2, k3, k4, k5, k6, k7, k8],
        [k2, k1, k8, k7, k6, k5, k4, k3],
        [k3, k8, k1, k6, k7, k4, k5, k2],
        [k4, k7, k6, k1, k8, k3, k2, k5],
        [k5, k6, k7, k8, k1, k2, k3, k4],
        [k6, k5, k4, k3, k2, k1, k8, k7],
        [k7, k4, k5, k2, k3, k8, k1, k6],
        [k8, k3, k2, k5, k4, k7, k6, k1]])
    # top88 orders nodes lower-left, lower-right, upper-right, upper-left with y pointing down
    # in its numbering; flip y and map to our lexicographic (x fastest, y up) local order.
    Ke = fem.element_stiffness(2, nu)
    # our local nodes: 0=(0,0) 1=(1,0) 2=(0,1) 3=(1,1).  top88 (y down): node A=(0,1)->(0,0) etc.
    perm_nodes = [2, 3, 1, 0]  # top88 node n sits at our local node perm_nodes[n] (y flipped)
    flip = np.array([1.0, -1.0])
    T = np.zeros((8, 8))
    for n, a in enumerate(perm_nodes):
        for c in range(2):
            T[2 * n + c, 2 * a + c] = flip[c]
    assert np.allclose(T @ Ke @ T.T, KE, atol=1e-15, rtol=0)


@pytest.mark.parametrize("dim,rank", [(2, 5), (3, 18)])
def test_ke_nullspace_rank_spd(dim, rank):
    Ke = fem.element_stiffness(dim, 0.3)
    assert np.abs(Ke - Ke.T).max() < 1e-15
    ev = np.linalg.eigvalsh(Ke)
    assert ev.min() > -1e-14
    assert np.linalg.matrix_rank(Ke, tol=1e-10) == rank
    coords = np.array([[(a >> k) & 1 for k in range(dim)] for a in range(1 << dim)], float)
    R = fem.rigid_body_modes(dim, coords)
    assert np.abs(Ke @ R).max() < 1e-14
    # translations: zero row sums per component
    for c in range(dim):
        assert np.abs(Ke[:, c::dim].sum(axis=1)).max() < 1e-15


def test_simp():
    assert fem.simp(0.0, 1.0, 1e-9, 3.0) == pytest.approx(1e-9, rel=0, abs=0)
    assert fem.simp(1.0, 1.0, 1e-9, 3.0) == 1.0
    assert fem.simp(0.5, 2.0, 0.0, 3.0) == 0.25
    assert fem.simp(0.5, 1.0, 1e-9, 3.0) == 1e-9 + (1.0 - 1e-9) * 0.125


def test_assembly_brute_force():
    """CSR assembly against an explicit element loop on a 3x2 grid with random E."""
    nx, ny = 3, 2
    rng = np.random.default_rng(0)
    E = rng.uniform(0.5, 2.0, nx * ny)
    Ke = fem.element_stiffness(2, 0.3)
    K = fem.assemble(2, nx, ny, 1, E, Ke).toarray()
    n = 2 * (nx + 1) * (ny + 1)
    Kb = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            nodes = [i + (nx + 1) * j, i + 1 + (nx + 1) * j, i + (nx + 1) * (j + 1), i + 1 + (nx + 1) * (j + 1)]
            dofs = [2 * nd + c for nd in nodes for c in range(2)]
            Kb[np.ix_(dofs, dofs)] += E[i + nx * j] * Ke
    assert np.allclose(K, Kb, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,grid", [(2, (2, 1, 1)), (2, (3, 2, 1)), (3, (2, 2, 2))])
def test_spd_after_bcs(dim, grid):
    p = W.random_problem(dim, *grid, seed=1, contrast="minmax")
    A = fem.masked_operator(fem.stiffness(p), p.fixed).toarray()
    assert np.abs(A - A.T).max() < 1e-15
    np.linalg.cholesky(A)
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("dim,grid", [(2, (16, 8, 1)), (3, (4, 4, 4))])
def test_direct_vs_dense(dim, grid):
    p = W.random_problem(dim, *grid, seed=2, contrast="minmax", nrhs=2)
    K = fem.stiffness(p)
    U = fem.direct_solve(K, p.fixed, p.f)
    free = fem.free_mask(p.n, p.fixed).astype(bool)
    Kd = K.toarray()[np.ix_(free, free)]
    for r in range(2):
        ud = np.linalg.solve(Kd, p.f[r, free])
        assert np.allclose(U[r, free], ud, rtol=1e-12, atol=1e-12 * np.abs(ud).max())
        assert np.all(U[r, ~free] == 0)
    # masked operator gives the same solution
    A = fem.masked_operator(K, p.fixed).toarray()
    m = fem.free_mask(p.n, p.fixed)
    um = np.linalg.solve(A, m * p.f[0])
    assert np.allclose(um, U[0], rtol=1e-10, atol=1e-12 * np.abs(um).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_uniform_tension(dim):
    sig, E, nu = 0.7, 2.5, 0.3
    p = W.patch_tension(dim, 5, 3, 2, sigma=sig, E=E, nu=nu)
    u = fem.direct_solve(fem.stiffness(p), p.fixed, p.f)[0]
    X = fem.node_coords(dim, p.nx, p.ny, p.nz)
    exact = np.zeros_like(X)
    exact[:, 0] = sig * X[:, 0] / E
    if dim == 2:
        exact[:, 1] = -nu * sig * X[:, 1] / E
    else:
        exact[:, 1] = -nu * sig * X[:, 1] / E
        exact[:, 2] = -nu * sig * X[:, 2] / E
    assert np.allclose(u.reshape(-1, dim), exact, rtol=0, atol=1e-12)


def test_compliance_and_scaling():
    p = W.random_problem(2, 12, 6, seed=3, contrast="minmax")
    K = fem.stiffness(p)
    u = fem.direct_solve(K, p.fixed, p.f)[0]
    c = fem.compliance(p.f[0], u)
    assert c > 0
    assert c == pytest.approx(u @ (K @ u), rel=1e-9)
    u2 = fem.direct_solve(4.0 * K, p.fixed, p.f)[0]
    assert np.allclose(u2, u / 4.0, rtol=1e-12, atol=0)
    assert fem.compliance(p.f[0], u2) == pytest.approx(c / 4.0, rel=1e-12)


def test_numbering_conventions():
    dofs = fem.element_dofs(3, 2, 3, 4)
    # element (i,j,k) = (1,2,3) -> e = 1 + 2*(2 + 3*3); local node 7 = (i+1, j+1, k+1)
    e = 1 + 2 * (2 + 3 * 3)
    node = 2 + 3 * (3 + 4 * 4)
    assert list(dofs[e, 21:24]) == [3 * node, 3 * node + 1, 3 * node + 2]


@pytest.mark.parametrize("dim,grid", [(2, (7, 5, 1)), (2, (1, 1, 1)), (3, (4, 3, 5)), (3, (1, 2, 1))])
def test_masked_apply_rows_matches_assembled(dim, grid):
    """The element-local row evaluation used for full-size checks equals the assembled masked
    operator on every node (corners, edges, faces and interior; fixed and free DOFs)."""
    nx, ny, nz = grid
    rng = np.random.default_rng(3)
    nn, nel, n = fem.grid_counts(dim, nx, ny, nz)
    E = 10.0 ** rng.uniform(-9, 0, nel)
    Ke = fem.element_stiffness(dim, 0.3)
    fixed = rng.choice(n, size=max(1, n // 5), replace=False)
    A = fem.masked_operator(fem.assemble(dim, nx, ny, nz, E, Ke), fixed)
    x = rng.standard_normal(n)
    rows = fem.masked_apply_rows(dim, nx, ny, nz, E, Ke, fixed, x, np.arange(nn))
    ref = (A @ x).reshape(nn, dim)
    assert np.abs(rows - ref).max() <= 1e-13 * np.abs(ref).max()
