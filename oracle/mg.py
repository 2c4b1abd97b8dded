"""Multigrid V-cycle and hierarchy builders (oracle, FP64, test use only).

V-cycle: Algorithm 1 (Sec. 3.2) with weighted point-block Jacobi smoothing (one block per node,
weight 0.5, Sec. 4.1) and a direct solve on the coarsest level.  Algorithm 1 as printed applies
(A^k)^-1 at the level whose successor is the coarsest; the reading adopted is the usual one:
levels 0..L-1, level L-1 is solved directly, every other level smooths, restricts with P^T,
recurses, prolongs with P and smooths again.  A one-level hierarchy is a direct solve.
The coarse direct solve is a dense Cholesky factorisation (the paper uses LU; the coarse
operator is SPD, Sec. 3.1), factored at setup (Sec. 3.2).

Hierarchies
  gmg     geometric levels from bilinear / trilinear P and Galerkin products (Sec. 3.2)
  amg     smoothed aggregation from the masked fine operator, rigid-body candidates (Sec. 4)
  hybrid  n_geo geometric levels, then smoothed aggregation from the last geometric operator
          with rigid-body modes evaluated at that level's node coordinates (Sec. 4.3, 4.4)

Parity: pinned (tests/test_oracle_mg.py: symmetric preconditioner, contraction < 1,
exactness of a one-level cycle, iteration counts bounded under refinement).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import fem, gmg, amg


@dataclass
class Hierarchy:
    A: list                       # CSR operators, level 0 = masked fine operator
    P: list                       # CSR prolongations, P[l]: level l+1 -> level l
    bs: list                      # DOFs per node (block size) on each level
    kinds: list                   # 'geo' or 'amg' per level
    omega: float = 0.5
    n_pre: int = 1
    n_post: int = 1
    block: bool = True
    Dinv: list = field(default_factory=list)
    chol: object = None
    info: dict = field(default_factory=dict)

    def finalize(self):
        self.Dinv = []
        for A, b in zip(self.A, self.bs):
            self.Dinv.append(amg.block_diag_inv(A, b if self.block else 1))
        Ac = self.A[-1].toarray()
        self.chol = sla.cho_factor(Ac, lower=True)
        return self

    @property
    def n_levels(self):
        return len(self.A)


def smooth(H, l, x, b):
    """One weighted (point-block) Jacobi sweep x + w D^-1 (b - A x)."""
    return x + H.omega * amg.apply_block_diag(H.Dinv[l], b - H.A[l] @ x)


def vcycle(H, b, l=0):
    """V-cycle multigrid, Algorithm 1 (reading stated in the module docstring)."""
    if l == H.n_levels - 1:
        return sla.cho_solve(H.chol, b)
    A = H.A[l]
    x = np.zeros_like(b)
    for _ in range(H.n_pre):
        x = smooth(H, l, x, b)
    bc = H.P[l].T @ (b - A @ x)
    x = x + H.P[l] @ vcycle(H, bc, l + 1)
    for _ in range(H.n_post):
        x = smooth(H, l, x, b)
    return x


def fine_operator(problem):
    K = fem.stiffness(problem)
    return fem.masked_operator(K, problem.fixed)


def build_gmg(problem, n_levels=None, cap=None, A0=None, finalize=True, **kw):
    p = problem
    if n_levels is None:
        n_levels = gmg.levels_for_cap(p.dim, p.nx, p.ny, p.nz, cap)
    A = [fine_operator(p) if A0 is None else A0]
    P = []
    g = (p.nx, p.ny, p.nz)
    for _ in range(n_levels - 1):
        Pl = gmg.prolongation(p.dim, *g)
        P.append(Pl)
        A.append(gmg.galerkin(A[-1], Pl))
        g = gmg.coarse_grid(p.dim, *g)
    H = Hierarchy(A, P, [p.dim] * n_levels, ["geo"] * n_levels, **kw)
    H.info["grids"] = gmg.grids(p.dim, p.nx, p.ny, p.nz, n_levels)
    return H.finalize() if finalize else H


def _sa_extend(H, B, cap, beta, max_levels):
    b = H.bs[-1]
    while H.A[-1].shape[0] >= cap and len(H.A) < max_levels:
        lev = amg.sa_level(H.A[-1], B, b, len(H.A) - 1, beta)
        if lev["n_agg"] == 0 or lev["P"].shape[1] >= H.A[-1].shape[0]:
            break
        H.P.append(lev["P"])
        H.A.append(lev["Ac"])
        H.bs.append(lev["k"])
        H.kinds.append("amg")
        H.info.setdefault("agg", []).append(lev["agg"])
        H.info.setdefault("omega_P", []).append(lev["omega"])
        B = lev["Bc"]
        b = lev["k"]
    return H


def build_amg(problem, cap, beta=0.003, max_levels=25, A0=None, **kw):
    p = problem
    A = [fine_operator(p) if A0 is None else A0]
    H = Hierarchy(A, [], [p.dim], ["geo"], **kw)
    B = fem.rigid_body_modes(p.dim, fem.node_coords(p.dim, p.nx, p.ny, p.nz))
    _sa_extend(H, B, cap, beta, max_levels)
    return H.finalize()


def build_hybrid(problem, n_geo, cap, beta=0.003, max_levels=25, A0=None, **kw):
    p = problem
    H = build_gmg(problem, n_levels=n_geo, A0=A0, finalize=False, **kw)
    g = H.info["grids"][-1]
    lvl = n_geo - 1
    xs = gmg.level_positions(p.nx, lvl)
    ys = gmg.level_positions(p.ny, lvl)
    zs = gmg.level_positions(p.nz, lvl) if p.dim == 3 else None
    B = fem.rigid_body_modes(p.dim, fem.node_coords(p.dim, g[0], g[1], g[2], xs, ys, zs))
    _sa_extend(H, B, cap, beta, max_levels)
    return H.finalize()
