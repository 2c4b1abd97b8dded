"""Textbook Krylov solvers (oracle, FP64, test use only).

* Preconditioned conjugate gradients (Hestenes & Stiefel 1952; the paper's CG, Sec. 3.1).
* Flexible CG (Notay 2000): beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k), the variant that
  tolerates a preconditioner that changes between iterations (the FP32 V-cycle).
  The paper's outer solver is GMRES (Sec. 4); CG/FCG is the reading adopted for the solve.

Stopping: ||b - A x||_2 / ||b||_2 <= rtol with the recursively updated residual, checked after
each update; the iteration count is the number of updates of x.  b = 0 returns x = 0 after
0 iterations.

Parity: pinned (tests/test_oracle_krylov.py: agreement with sparse direct solves, exact
convergence in n steps on tiny SPD systems, FCG = PCG for a fixed SPD preconditioner).
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, M=None, x0=None, rtol=1e-8, max_iter=1000, flexible=False):
    """Returns (x, iterations, relative residual history)."""
    M = (lambda r: r.copy()) if M is None else M
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - A @ x
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < max_iter:
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            break
        z = M(r)
        rz_new = r @ z
        beta = (z @ (r - r_old)) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist
