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

Smoothers
  jacobi     weighted point-block Jacobi x + w D^-1 (b - A x), n_pre / n_post sweeps
  chebyshev  point-block-Jacobi-preconditioned Chebyshev polynomial of degree m (the paper
             studies a Chebyshev smoother beside Jacobi, Sec. 4.1; its SOR preconditioning is a
             sequential sweep and is replaced by the point-block diagonal).  The polynomial is
             the Chebyshev polynomial of D^-1 A on [lower, upper] * lambda, lambda from 20
             power iterations (the estimate also used to smooth AMG prolongators), written as
             the three-term recurrence of Chebyshev acceleration (Saad, Iterative Methods for
             Sparse Linear Systems, 2nd ed., Alg. 12.1).  Pre- and post-smoothing use the same
             polynomial, so the cycle stays symmetric.
  gmres      m steps of right-preconditioned GMRES (Saad, Alg. 9.5) with the point-block
             diagonal in place of the paper's SOR preconditioning (Sec. 4.1 studies an
             SOR-preconditioned GMRES smoother under flexible GMRES): Arnoldi by modified
             Gram-Schmidt from r_0 = b - A x_0, the least-squares problem
             min ||beta e_1 - Hbar y|| solved by a library routine, x = x_0 + D^-1 V y.  An exact
             breakdown (a zero new Arnoldi vector, r_0 = 0 included) ends the steps early.  The
             smoother depends nonlinearly on its right-hand side, so the cycle is a variable
             preconditioner and needs a flexible outer method (FCG or FGMRES).

Parity: pinned (tests/test_oracle_mg.py: symmetric preconditioner, contraction < 1,
exactness of a one-level cycle, iteration counts bounded under refinement; the Chebyshev
smoother's error propagation equals the scaled Chebyshev polynomial evaluated by
numpy.polynomial.chebyshev on every eigenvector of D^-1 A; the GMRES smoother's result
against the minimiser of ||b - A x|| over the explicit power basis of the preconditioned
Krylov space, finite termination at m = n, exact breakdowns).
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
    smoother: str = "jacobi"      # or "chebyshev", "gmres"
    cheb_degree: int = 2
    gmres_steps: int = 2          # GMRES smoother: Arnoldi steps per smoothing
    cheb_lower: float = 0.1       # interval [lower, upper] * lambda(D^-1 A)
    cheb_upper: float = 1.1
    Dinv: list = field(default_factory=list)
    lam: list = field(default_factory=list)
    chol: object = None
    info: dict = field(default_factory=dict)

    def finalize(self):
        self.Dinv = []
        for A, b in zip(self.A, self.bs):
            self.Dinv.append(amg.block_diag_inv(A, b if self.block else 1))
        self.lam = []
        if self.smoother == "chebyshev":
            for l in range(self.n_levels - 1):
                self.lam.append(amg.spectral_radius_DinvA(self.A[l], self.Dinv[l], l))
        Ac = self.A[-1].toarray()
        self.chol = sla.cho_factor(Ac, lower=True)
        return self

    @property
    def n_levels(self):
        return len(self.A)


def smooth(H, l, x, b):
    """One weighted (point-block) Jacobi sweep x + w D^-1 (b - A x)."""
    return x + H.omega * amg.apply_block_diag(H.Dinv[l], b - H.A[l] @ x)


def chebyshev_coefficients(lam_lo, lam_hi, m):
    """Step coefficients of Chebyshev acceleration on [lam_lo, lam_hi] (Saad, Alg. 12.1):
    d_0 = c2_0 D^-1 r_0 and d_k = c1_k d_{k-1} + c2_k D^-1 r_k, with theta = centre,
    delta = half width, sigma = theta / delta, rho_0 = 1 / sigma,
    rho_k = 1 / (2 sigma - rho_{k-1}), c1_k = rho_k rho_{k-1}, c2_k = 2 rho_k / delta."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    c1, c2 = [0.0], [1.0 / theta]
    for _ in range(1, m):
        rho_new = 1.0 / (2.0 * sigma - rho)
        c1.append(rho_new * rho)
        c2.append(2.0 * rho_new / delta)
        rho = rho_new
    return c1, c2


def chebyshev_smooth(A, Dinv, x, b, lam_lo, lam_hi, m):
    """m steps of Chebyshev acceleration for A x = b preconditioned by the point-block
    diagonal: x_{k+1} = x_k + d_k, d_k from the residual r_k = b - A x_k (m applies of A)."""
    c1, c2 = chebyshev_coefficients(lam_lo, lam_hi, m)
    d = np.zeros_like(x)
    for k in range(m):
        r = b - A @ x
        d = c1[k] * d + c2[k] * amg.apply_block_diag(Dinv, r)
        x = x + d
    return x


def gmres_smooth(A, Dinv, x, b, m):
    """m steps of GMRES for A x = b from x, right-preconditioned by the point-block diagonal
    (Saad, Alg. 9.5): Arnoldi on A D^-1 by modified Gram-Schmidt, then the small
    least-squares problem; stops early at an exact breakdown."""
    r = b - A @ x
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x
    Vb = [r / beta]
    Z = []
    Hb = np.zeros((m + 1, m))
    k = 0
    for j in range(m):
        z = amg.apply_block_diag(Dinv, Vb[j])
        Z.append(z)
        w = A @ z
        for i in range(j + 1):
            Hb[i, j] = w @ Vb[i]
            w = w - Hb[i, j] * Vb[i]
        Hb[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        if Hb[j + 1, j] == 0.0:
            break
        Vb.append(w / Hb[j + 1, j])
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y = np.linalg.lstsq(Hb[:k + 1, :k], e1, rcond=None)[0]
    for i in range(k):
        x = x + y[i] * Z[i]
    return x


def presmooth(H, l, b):
    if H.smoother == "gmres":
        return gmres_smooth(H.A[l], H.Dinv[l], np.zeros_like(b), b, H.gmres_steps)
    if H.smoother == "chebyshev":
        lam = H.lam[l]
        return chebyshev_smooth(H.A[l], H.Dinv[l], np.zeros_like(b), b, H.cheb_lower * lam,
                                H.cheb_upper * lam, H.cheb_degree)
    x = np.zeros_like(b)
    for _ in range(H.n_pre):
        x = smooth(H, l, x, b)
    return x


def postsmooth(H, l, x, b):
    if H.smoother == "gmres":
        return gmres_smooth(H.A[l], H.Dinv[l], x, b, H.gmres_steps)
    if H.smoother == "chebyshev":
        lam = H.lam[l]
        return chebyshev_smooth(H.A[l], H.Dinv[l], x, b, H.cheb_lower * lam, H.cheb_upper * lam,
                                H.cheb_degree)
    for _ in range(H.n_post):
        x = smooth(H, l, x, b)
    return x


def vcycle(H, b, l=0):
    """V-cycle multigrid, Algorithm 1 (reading stated in the module docstring)."""
    if l == H.n_levels - 1:
        return sla.cho_solve(H.chol, b)
    A = H.A[l]
    x = presmooth(H, l, b)
    bc = H.P[l].T @ (b - A @ x)
    x = x + H.P[l] @ vcycle(H, bc, l + 1)
    return postsmooth(H, l, x, b)


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
