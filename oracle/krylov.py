"""Textbook Krylov solvers (oracle, FP64, test use only).

* Preconditioned conjugate gradients (Hestenes & Stiefel 1952; the paper's CG, Sec. 3.1).
* Flexible CG (Notay 2000): beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k), the variant that
  tolerates a preconditioner that changes between iterations (the FP32 V-cycle).
  The paper's outer solver is GMRES (Sec. 4); CG/FCG is the reading adopted for the solve.
* Flexible GMRES(m) (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Alg. 9.6):
  right-preconditioned Arnoldi with modified Gram-Schmidt, the preconditioned vectors kept
  (z_j = M v_j), Givens rotations for the least-squares problem, restart after m steps.  The
  paper's outer solver (GMRES with the MG preconditioner, FGMRES with a GMRES smoother, Sec. 4).

Stopping: ||b - A x||_2 / ||b||_2 <= rtol with the recursively updated residual, checked after
each update; the iteration count is the number of updates of x.  b = 0 returns x = 0 after
0 iterations.

Parity: pinned (tests/test_oracle_mg.py: agreement with sparse direct solves, exact
convergence in n steps on tiny SPD systems, FCG = PCG for a fixed SPD preconditioner; FGMRES:
the minimal-residual property against a brute-force least-squares solve over the explicit
Krylov basis, finite termination, non-increasing residuals).
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


def fgmres(A, b, M=None, x0=None, rtol=1e-8, max_iter=1000, restart=30):
    """Flexible GMRES(m).  Returns (x, iterations, residual estimate history); the iteration
    count is the number of Arnoldi steps (preconditioner applications).  Every cycle starts
    from the true residual b - A x; the run stops when the true relative residual is within
    rtol at the end of a cycle (the cycle ends early once the Givens estimate is within)."""
    M = (lambda r: r.copy()) if M is None else M
    n = b.size
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    it = 0
    hist = []
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta / nb <= rtol or it >= max_iter:
            return x, it, hist
        m = restart
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = A @ Z[:, j]
            for i in range(j + 1):
                H[i, j] = w @ V[:, i]
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            # previous rotations, then the one that annihilates H[j+1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / nb)
            if hist[-1] <= rtol or it >= max_iter:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:, :k] @ y
