"""Finite-element pieces of the SIMP elasticity system K(rho) u = f (oracle, FP64, test use only).

* SIMP interpolation E(rho) = Emin + (E0 - Emin) rho^p                      (Sec. 2.1, Eq. 2)
* compliance f^T u                                                           (Sec. 2.1, Eq. 1)
* K symmetric positive definite after boundary conditions; direct solve      (Sec. 3.1)
* element stiffness: bilinear quad4 (plane stress) / trilinear hex8 on the unit element,
  Ke = integral of B^T D B, 2x2(x2) Gauss rule.  The paper names uniform bilinear quadrilateral
  and trilinear hexahedral elements only; the plane-stress / isotropic D and nu are the
  readings adopted project-wide.

Local node a of an element has bits (a_x, a_y, a_z) = (a & 1, a >> 1 & 1, a >> 2 & 1) and sits at
global node (i + a_x, j + a_y, k + a_z); local DOF = d * a + c.

Boundary conditions use the masked operator A = M K M + (I - M) (M = diag of the free-DOF mask),
whose solution on free DOFs equals the eliminated system's and is 0 on fixed DOFs.

Parity: pinned (tests/test_oracle_fem.py: exact rational integration, textbook quad4 matrix,
rigid-body null space, rank, patch test, scaling, SPD, dense solves).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def simp(rho, E0, Emin, penal):
    """Modified SIMP interpolation E = Emin + (E0 - Emin) * rho^p (Sec. 2.1)."""
    rho = np.asarray(rho, dtype=np.float64)
    return Emin + (E0 - Emin) * rho ** penal


def constitutive(dim, E, nu):
    """Plane-stress D (3x3, strains [exx, eyy, gxy]) or 3D isotropic D (6x6, strains
    [exx, eyy, ezz, gyz, gxz, gxy])."""
    if dim == 2:
        c = E / (1.0 - nu * nu)
        return c * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]])
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_grad(dim, xi):
    """Gradients dN_a/dxi_k of the 2^dim multilinear shape functions at point xi in [0,1]^dim.
    Returns an array (2^dim, dim)."""
    nn = 1 << dim
    G = np.zeros((nn, dim))
    for a in range(nn):
        bits = [(a >> k) & 1 for k in range(dim)]
        for k in range(dim):
            g = 1.0 if bits[k] else -1.0
            for m in range(dim):
                if m != k:
                    g *= xi[m] if bits[m] else (1.0 - xi[m])
            G[a, k] = g
    return G


def strain_matrix(dim, G):
    """Strain-displacement matrix B from shape-function gradients G (2^dim, dim)."""
    nn = G.shape[0]
    if dim == 2:
        B = np.zeros((3, 2 * nn))
        for a in range(nn):
            nx_, ny_ = G[a]
            B[0, 2 * a] = nx_
            B[1, 2 * a + 1] = ny_
            B[2, 2 * a] = ny_
            B[2, 2 * a + 1] = nx_
        return B
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        gx, gy, gz = G[a]
        c = 3 * a
        B[0, c] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1] = gz
        B[3, c + 2] = gy
        B[4, c] = gz
        B[4, c + 2] = gx
        B[5, c] = gy
        B[5, c + 1] = gx
    return B


def element_stiffness(dim, nu, E=1.0):
    """Ke = sum over the 2x2(x2) Gauss points on [0,1]^dim of w B^T D B (unit element)."""
    g = [0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)]
    D = constitutive(dim, E, nu)
    nd = dim * (1 << dim)
    Ke = np.zeros((nd, nd))
    w = 0.5 ** dim
    for p in range(1 << dim):
        xi = [g[(p >> k) & 1] for k in range(dim)]
        B = strain_matrix(dim, shape_grad(dim, xi))
        Ke += w * B.T @ D @ B
    return Ke


def grid_counts(dim, nx, ny, nz):
    nn = (nx + 1) * (ny + 1) * ((nz + 1) if dim == 3 else 1)
    nel = nx * ny * (nz if dim == 3 else 1)
    return nn, nel, dim * nn


def element_dofs(dim, nx, ny, nz):
    """(Nel, dim * 2^dim) global DOF indices of every element in local DOF order."""
    if dim == 2:
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), np.zeros(nx * ny, dtype=np.int64)
    else:
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
    cols = []
    for a in range(1 << dim):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        node = (i + ax) + (nx + 1) * ((j + ay) + (ny + 1) * (k + az))
        for c in range(dim):
            cols.append(dim * node + c)
    return np.stack(cols, axis=1).astype(np.int64)


def assemble(dim, nx, ny, nz, E, Ke, chunk=1 << 19):
    """K = sum_e E_e * Ke scattered to global DOFs, as a scipy CSR matrix (Sec. 2.1, 3.1).
    The sum runs over consecutive groups of at most ``chunk`` elements, each group scattered
    and added to K (the same sum; it only bounds the host memory of the scatter on grids of
    millions of elements)."""
    _, nel, n = grid_counts(dim, nx, ny, nz)
    edofs = element_dofs(dim, nx, ny, nz)
    nd = edofs.shape[1]
    E = np.asarray(E, dtype=np.float64)
    K = None
    for e0 in range(0, nel, chunk):
        ed = edofs[e0:e0 + chunk]
        rows = np.repeat(ed, nd, axis=1).ravel()
        cols = np.tile(ed, (1, nd)).ravel()
        vals = (E[e0:e0 + chunk, None] * Ke.ravel()[None, :]).ravel()
        part = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
        part.sum_duplicates()
        del rows, cols, vals
        K = part if K is None else (K + part).tocsr()
    K.sum_duplicates()
    return K


def masked_apply_rows(dim, nx, ny, nz, E, Ke, fixed, x, nodes):
    """(A x) at every DOF of the given nodes, A = M K M + (I - M), without assembling K: each
    node sums E_e Ke[local rows] x_e over the (up to 2^dim) elements around it (Sec. 2.1, 3.1).
    For checks at sizes where assembling K is too large.  Returns (len(nodes), dim)."""
    n = dim * (nx + 1) * (ny + 1) * ((nz + 1) if dim == 3 else 1)
    m = free_mask(n, fixed)
    xm = x * m
    out = np.zeros((len(nodes), dim))
    for t, node in enumerate(np.asarray(nodes, dtype=np.int64)):
        i = node % (nx + 1)
        j = (node // (nx + 1)) % (ny + 1)
        k = node // ((nx + 1) * (ny + 1)) if dim == 3 else 0
        acc = np.zeros(dim)
        for a in range(1 << dim):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            ei, ej, ek = i - ax, j - ay, k - az  # element whose local node a is this node
            if ei < 0 or ei >= nx or ej < 0 or ej >= ny or (dim == 3 and (ek < 0 or ek >= nz)):
                continue
            e = ei + nx * (ej + ny * ek)
            dofs = []
            for b in range(1 << dim):
                bx, by, bz = b & 1, (b >> 1) & 1, (b >> 2) & 1
                nb = (ei + bx) + (nx + 1) * ((ej + by) + (ny + 1) * (ek + bz))
                dofs += [dim * nb + c for c in range(dim)]
            acc += E[e] * (Ke[dim * a:dim * a + dim, :] @ xm[dofs])
        d = dim * node + np.arange(dim)
        out[t] = m[d] * acc + (1.0 - m[d]) * x[d]
    return out


def free_mask(n, fixed):
    m = np.ones(n, dtype=np.float64)
    m[np.asarray(fixed, dtype=np.int64)] = 0.0
    return m


def masked_operator(K, fixed):
    """A = M K M + (I - M): identity rows/columns on fixed DOFs, K elsewhere.  Entry (i, j) of
    K is scaled by m_i m_j in place of the two diagonal products, and the diagonal entries of
    fixed DOFs (present in K, every DOF belongs to an element) are set to 1."""
    m = free_mask(K.shape[0], fixed)
    A = K.tocsr(copy=True)
    A.sum_duplicates()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    A.data *= m[rows] * m[A.indices]
    del rows
    fx = np.flatnonzero(m == 0.0)
    if fx.size:
        A[fx, fx] = 1.0
    A.eliminate_zeros()
    return A


def stiffness(problem):
    """Assembled K (CSR) of a :class:`workloads.Problem`."""
    p = problem
    Ke = element_stiffness(p.dim, p.nu)
    E = simp(p.rho, p.E0, p.Emin, p.penal)
    return assemble(p.dim, p.nx, p.ny, p.nz, E, Ke)


def direct_solve(K, fixed, f, refine=3):
    """u = K_ff^{-1} f_f, u_fixed = 0, by sparse LU of the reduced system (Sec. 3.1 direct
    solver; SuperLU via scipy), followed by iterative refinement with the same factors
    (Wilkinson): r = f - K u, u += LU^{-1} r, at most ``refine`` times, until the correction is
    below 1e-14 of u.  With a 1e9 stiffness contrast the unrefined LU solution is off by about
    1e-6 (relative) although its residual is below 1e-8; refinement brings it to the accuracy
    FP64 allows.  ``f`` is (n,) or (nrhs, n)."""
    n = K.shape[0]
    free = free_mask(n, fixed).astype(bool)
    Kff = K[free][:, free].tocsc()
    lu = spla.splu(Kff)
    F = np.atleast_2d(f)
    U = np.zeros_like(F, dtype=np.float64)
    for r in range(F.shape[0]):
        b = F[r, free]
        u = lu.solve(b)
        for _ in range(refine):
            du = lu.solve(b - Kff @ u)
            u = u + du
            if np.linalg.norm(du) <= 1e-14 * np.linalg.norm(u):
                break
        U[r, free] = u
    return U.reshape(np.shape(f))


def compliance(f, u):
    """c = f^T u (Sec. 2.1, Eq. 1), per right-hand side."""
    return np.einsum("...i,...i->...", np.asarray(f), np.asarray(u))


def node_coords(dim, nx, ny, nz, xs=None, ys=None, zs=None):
    """(nn, dim) coordinates of the grid nodes; optional per-axis position arrays
    (coarse geometric levels sit at a subset of fine positions)."""
    xs = np.arange(nx + 1, dtype=np.float64) if xs is None else np.asarray(xs, np.float64)
    ys = np.arange(ny + 1, dtype=np.float64) if ys is None else np.asarray(ys, np.float64)
    if dim == 2:
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        return np.stack([X.ravel(), Y.ravel()], axis=1)
    zs = np.arange(nz + 1, dtype=np.float64) if zs is None else np.asarray(zs, np.float64)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def rigid_body_modes(dim, coords):
    """Near-nullspace candidates: rigid translations and infinitesimal rotations evaluated at
    the node coordinates, before boundary conditions (Sec. 4 AMG setup).  3 modes in 2D
    [tx, ty, rz], 6 in 3D [tx, ty, tz, rx, ry, rz]; interleaved DOF rows (n, k)."""
    nn = coords.shape[0]
    if dim == 2:
        B = np.zeros((2 * nn, 3))
        x, y = coords[:, 0], coords[:, 1]
        B[0::2, 0] = 1.0
        B[1::2, 1] = 1.0
        B[0::2, 2] = -y
        B[1::2, 2] = x
        return B
    B = np.zeros((3 * nn, 6))
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    B[0::3, 0] = 1.0
    B[1::3, 1] = 1.0
    B[2::3, 2] = 1.0
    # rotation about x: (0, -z, y); about y: (z, 0, -x); about z: (-y, x, 0)
    B[1::3, 3] = -z
    B[2::3, 3] = y
    B[0::3, 4] = z
    B[2::3, 4] = -x
    B[0::3, 5] = -y
    B[1::3, 5] = x
    return B
