"""Geometric multigrid pieces (oracle, FP64, test use only).

* Prolongation P from the shape functions of the next-coarser grid: bilinear / trilinear
  interpolation with 2x coarsening per axis (Sec. 3.2, "defined by shape function values on
  the coarse grids").  The paper is silent on odd element counts; the reading adopted is
  ceil(n/2) coarse elements per axis with coarse node I at fine position min(2I, n), i.e. the
  last coarse element spans a single fine element when n is odd.  This reproduces the paper's
  5-level coarse grid of 2312 DOFs for the 520 x 520 grid (Sec. 4.3).
* Galerkin coarse operators A^{l+1} = P^T A^l P, R = P^T (Sec. 3.2, Eq. 9).
* Level count from a coarse-size cap: the fewest levels (fine grid included) whose coarsest
  grid has fewer DOFs than the cap (reproduces 9/6/5 levels for caps 150/5000/20000 on
  2048 x 1024, Sec. 4.1).

Parity: pinned (tests/test_oracle_gmg.py: the paper's coarse-DOF numbers, linear-field
reproduction, dense P^T A P).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def coarse_count(n):
    """Coarse elements along an axis with n fine elements."""
    return (n + 1) // 2


def coarse_positions(n):
    """Fine-grid positions of the coarse nodes along an axis with n fine elements."""
    nc = coarse_count(n)
    return np.minimum(2 * np.arange(nc + 1), n)


def prolong_1d(n):
    """(n+1) x (nc+1) 1D linear interpolation matrix from coarse to fine nodes."""
    pos = coarse_positions(n)
    nc = len(pos) - 1
    P = np.zeros((n + 1, nc + 1))
    for I, p in enumerate(pos):
        P[p, I] = 1.0
    for I in range(nc):
        a, b = pos[I], pos[I + 1]
        for p in range(a + 1, b):
            t = (p - a) / (b - a)
            P[p, I] = 1.0 - t
            P[p, I + 1] = t
    return P


def prolongation(dim, nx, ny, nz):
    """DOF prolongation P = (P_z (x) P_y (x) P_x) (x) I_dim for the interleaved numbering."""
    Pn = sp.kron(sp.csr_matrix(prolong_1d(ny)), sp.csr_matrix(prolong_1d(nx)))
    if dim == 3:
        Pn = sp.kron(sp.csr_matrix(prolong_1d(nz)), Pn)
    return sp.kron(Pn, sp.identity(dim)).tocsr()


def coarse_grid(dim, nx, ny, nz):
    return (coarse_count(nx), coarse_count(ny), coarse_count(nz) if dim == 3 else 1)


def grid_dofs(dim, nx, ny, nz):
    return dim * (nx + 1) * (ny + 1) * ((nz + 1) if dim == 3 else 1)


def levels_for_cap(dim, nx, ny, nz, cap, max_levels=30):
    """Fewest levels (fine level included) such that the coarsest grid has < cap DOFs."""
    L = 1
    g = (nx, ny, nz)
    while grid_dofs(dim, *g) >= cap and L < max_levels:
        ng = coarse_grid(dim, *g)
        if ng == g:
            break
        g = ng
        L += 1
    return L


def grids(dim, nx, ny, nz, n_levels):
    """Element counts (nx, ny, nz) of levels 0..n_levels-1."""
    out = [(nx, ny, nz if dim == 3 else 1)]
    for _ in range(n_levels - 1):
        out.append(coarse_grid(dim, *out[-1]))
    return out


def level_positions(n, level):
    """Fine-grid coordinates of the nodes of geometric level ``level`` along one axis."""
    pos = np.arange(n + 1)
    m = n
    for _ in range(level):
        pos = pos[coarse_positions(m)]
        m = coarse_count(m)
    return pos.astype(np.float64)


def galerkin(A, P):
    """A_c = P^T A P (Eq. 9)."""
    return (P.T @ A @ P).tocsr()
