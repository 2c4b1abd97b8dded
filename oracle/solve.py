"""One-call oracle solve mirroring the library's options (test use only).

The method reaches the unique solution of K(rho) u = f with u = 0 on fixed DOFs (K SPD after
boundary conditions, Sec. 3.1); ``direct`` computes that definition by sparse LU, ``solve``
runs the textbook PCG / FCG with the chosen multigrid preconditioner, and both return the
compliance f^T u (Eq. 1).

Parity: pinned through the modules it calls.
"""
from __future__ import annotations

import numpy as np

from . import fem, mg, krylov


def direct(problem):
    K = fem.stiffness(problem)
    U = fem.direct_solve(K, problem.fixed, problem.f)
    return dict(u=U, compliance=fem.compliance(problem.f, U))


def build(problem, pc="gmg", n_levels=None, cap=None, n_geo=None, beta=0.003, omega=0.5,
          A0=None, smoother="jacobi", cheb_degree=2, cheb_lower=0.1, cheb_upper=1.1,
          gmres_steps=2):
    kw = dict(omega=omega, smoother=smoother, cheb_degree=cheb_degree, cheb_lower=cheb_lower,
              cheb_upper=cheb_upper, gmres_steps=gmres_steps)
    if pc == "gmg":
        return mg.build_gmg(problem, n_levels=n_levels, cap=cap, A0=A0, **kw)
    if pc == "amg":
        return mg.build_amg(problem, cap=cap, beta=beta, A0=A0, **kw)
    if pc == "hybrid":
        return mg.build_hybrid(problem, n_geo=n_geo, cap=cap, beta=beta, A0=A0, **kw)
    raise ValueError(pc)


def solve(problem, pc="gmg", rtol=1e-8, max_iter=1000, flexible=False, x0=None, H=None,
          krylov_method="cg", restart=30, **kw):
    """Solve every right-hand side of ``problem``; returns a dict of stacked results.
    krylov_method: "cg" (PCG, or flexible CG with flexible=True; always flexible with the GMRES
    smoother, a variable preconditioner) or "fgmres" (FGMRES(restart))."""
    A0 = mg.fine_operator(problem)
    if H is None:
        H = build(problem, pc=pc, A0=A0, **kw)
    if H.smoother == "gmres":
        flexible = True
    m = fem.free_mask(problem.n, problem.fixed)
    F = np.atleast_2d(problem.f)
    U = np.zeros_like(F)
    its, rel = [], []
    for r in range(F.shape[0]):
        b = m * F[r]
        x0r = None if x0 is None else np.atleast_2d(x0)[r]
        if krylov_method == "fgmres":
            x, it, hist = krylov.fgmres(A0, b, M=lambda v: mg.vcycle(H, v), x0=x0r, rtol=rtol,
                                        max_iter=max_iter, restart=restart)
        else:
            x, it, hist = krylov.pcg(A0, b, M=lambda v: mg.vcycle(H, v), x0=x0r, rtol=rtol,
                                     max_iter=max_iter, flexible=flexible)
        U[r] = x
        its.append(it)
        nb = np.linalg.norm(b)
        rel.append(np.linalg.norm(b - A0 @ x) / nb if nb > 0 else 0.0)
    return dict(u=U, iterations=np.array(its), rel_residual=np.array(rel),
                compliance=fem.compliance(F, U), H=H)
