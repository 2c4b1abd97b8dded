"""Pins for oracle.gmg: the paper's printed coarse-grid sizes, interpolation, Galerkin products."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem, gmg

GOLD = os.path.join(os.path.dirname(__file__), "golden", "coarse_dofs.txt")


def _rows():
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            yield tuple(int(v) for v in line.split())


@pytest.mark.parametrize("row", list(_rows()))
def test_paper_coarse_sizes(row):
    dim, nx, ny, nz, cap, levels, dofs = row
    g = gmg.grids(dim, nx, ny, nz, levels)[-1]
    assert gmg.grid_dofs(dim, *g) == dofs
    if cap:
        assert gmg.levels_for_cap(dim, nx, ny, nz, cap) == levels


def test_fine_dof_count_appendix():
    # "approximately 100e6" DOFs for 512x256x256 (Appendix)
    assert gmg.grid_dofs(3, 512, 256, 256, ) == 3 * 513 * 257 * 257 == 101_649_411


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 33])
def test_prolong_1d_linear_and_partition(n):
    P = gmg.prolong_1d(n)
    pos = gmg.coarse_positions(n)
    assert np.allclose(P.sum(axis=1), 1.0)
    xf = np.arange(n + 1, dtype=float)
    assert np.allclose(P @ pos.astype(float), xf)
    assert pos[0] == 0 and pos[-1] == n and len(pos) == gmg.coarse_count(n) + 1
    assert set(np.unique(P)) <= {0.0, 0.5, 1.0}


@pytest.mark.parametrize("dim,grid", [(2, (5, 4, 1)), (2, (7, 3, 1)), (3, (3, 4, 5))])
def test_prolongation_reproduces_linear_fields(dim, grid):
    nx, ny, nz = grid
    P = gmg.prolongation(dim, nx, ny, nz)
    cg = gmg.coarse_grid(dim, nx, ny, nz)
    Xf = fem.node_coords(dim, nx, ny, nz)
    Xc = fem.node_coords(dim, *cg, xs=gmg.coarse_positions(nx), ys=gmg.coarse_positions(ny),
                         zs=gmg.coarse_positions(nz) if dim == 3 else None)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((dim, dim))
    t = rng.standard_normal(dim)
    uc = (Xc @ G.T + t).ravel()
    uf = (Xf @ G.T + t).ravel()
    assert np.allclose(P @ uc, uf, atol=1e-12)


@pytest.mark.parametrize("dim,grid", [(2, (5, 3, 1)), (3, (3, 2, 3))])
def test_galerkin_vs_dense(dim, grid):
    p = W.random_problem(dim, *grid, seed=4, contrast="minmax")
    A = fem.masked_operator(fem.stiffness(p), p.fixed)
    P = gmg.prolongation(dim, p.nx, p.ny, p.nz)
    Ac = gmg.galerkin(A, P).toarray()
    Pd, Ad = P.toarray(), A.toarray()
    ref = Pd.T @ Ad @ Pd
    assert np.allclose(Ac, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.linalg.eigvalsh(Ac).min() > 0


def test_uniform_coarse_operator_rigid_nullspace():
    nx, ny = 8, 4
    Ke = fem.element_stiffness(2, 0.3)
    K = fem.assemble(2, nx, ny, 1, np.ones(nx * ny), Ke)
    P = gmg.prolongation(2, nx, ny, 1)
    Kc = gmg.galerkin(K, P)
    cg = gmg.coarse_grid(2, nx, ny, 1)
    Xc = fem.node_coords(2, *cg, xs=gmg.coarse_positions(nx), ys=gmg.coarse_positions(ny))
    R = fem.rigid_body_modes(2, Xc)
    assert np.abs(Kc @ R).max() < 1e-12


def test_level_positions():
    assert list(gmg.level_positions(5, 1)) == [0, 2, 4, 5]
    assert list(gmg.level_positions(5, 2)) == [0, 4, 5]
    assert list(gmg.level_positions(8, 3)) == [0, 8]
