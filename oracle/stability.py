"""Linear buckling (stability) eigenproblem K_sigma Phi = lambda K Phi and the generalized
Davidson eigensolver (oracle, FP64, test infrastructure only).

Stress stiffness (Sec. 2.2, Eq. 4-5).  The pre-buckling stress of element e is evaluated at the
element centre from the displacements u of K u = f:
    sigma_e = E_sigma(rho_e) D_0 B(centre) u_e,   E_sigma(rho) = E0 rho^p if rho >= 0.1 else 0,
with D_0 the unit-modulus constitutive matrix.  With S_e the d x d stress tensor and
L_ij[a, b] = integral over the unit element of dN_a/dx_i dN_b/dx_j, the element geometric
stiffness is K_G,e = (sum_ij S_e,ij L_ij) (x) I_d (one copy per displacement component).  The
paper writes the eigenproblem as K_sigma Phi = lambda K Phi with lambda_max = 1 / P_critical;
the reading adopted is K_sigma = -K_G, so that compression gives positive lambda = 1 / mu for
the load factors mu of (K + mu K_G) Phi = 0.  Fixed DOFs: K_sigma is masked (M K_sigma M),
K is the masked operator M K M + (I - M) of the solve.

Generalized Davidson (Sec. 3.3, Algorithm 2): a K-orthonormal search space V of j_min..j_max
vectors; Rayleigh-Ritz on V (the projected matrix V^T K_sigma V, V^T K V = I); the largest
Ritz pairs are the targets; the search space grows by the preconditioned residual
z = M(K_sigma q - theta K q) of the largest unconverged pair, orthonormalised against V, and
is reset to the j_min best Ritz vectors when it reaches j_max.  The paper's settings:
j_min = 10, j_max = 25, six modes.  Start vectors: splitmix64 uniform vectors.

Sensitivities (Sec. 2.2, Eq. 6-9).  For a K-normalised mode (Phi^T K Phi = 1):
    dlambda/drho_e = E_sigma'(rho_e) Phi_e^T K_sigma,e^1 Phi_e - lambda E'(rho_e) Phi_e^T Ke Phi_e
                     - E'(rho_e) v_e^T Ke u_e,          K v = g = d(Phi^T K_sigma(u) Phi)/du,
with K_sigma,e^1 the element stress stiffness for a unit stress modulus, E' the derivative of
the SIMP modulus of K (Eq. 2) and E_sigma' that of Eq. 5 (0 below the cutoff).  The adjoint
term follows from u = u(rho): d(Phi^T K_sigma Phi) picks up g^T du/drho_e and
du/drho_e = -K^-1 (dK/drho_e) u.  The paper prints that term as +v^T E_sigma' (dK/dE) u; the
reading adopted is the derivation's -v^T E' (dK/dE) u (the modulus of K is E, not E_sigma; the
sign is that of v solving K v = g as printed), which central finite differences of the dense
eigenvalues confirm.  K_sigma is linear in u, so g does not depend on u:
    g = -sum_e E_sigma(rho_e) B^T D_0 w_e(Phi),   w_e,v = sum_ab L_ij[a, b] Phi_a . Phi_b
summed over the index pairs (i, j) of Voigt component v (both orders for a shear component),
masked at fixed DOFs.  The objective aggregates the n largest eigenvalues by a p-norm
(p = 8, n = 6): F = (sum_i lambda_i^p)^(1/p), dF/drho = F^(1-p) sum_i lambda_i^(p-1) dlambda_i/drho.

Parity: pinned (tests/test_oracle_stability.py: L_ij against exact rational integration,
symmetry and the translation null space of K_sigma, the stresses of constant-strain fields,
Davidson eigenvalues against dense scipy.linalg.eigh on small grids, the critical load of a
slender fixed-free column against Euler's formula, the adjoint right-hand side against
Phi^T K_sigma(e_i) Phi for every unit displacement e_i, the eigenvalue and p-norm
sensitivities against central finite differences of dense generalized eigenvalues).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .hashing import SALT_POWER, unit_uniform

SALT_GD = SALT_POWER + 1000  # start vector k of the Davidson search space uses salt SALT_GD + k


def stress_interp(rho, E0, penal, cutoff=0.1):
    """E_sigma(rho) = E0 rho^p for rho >= cutoff, else 0 (Eq. 5)."""
    rho = np.asarray(rho, dtype=np.float64)
    return np.where(rho >= cutoff, E0 * rho ** penal, 0.0)


def gradient_products(dim):
    """L[i][j] = integral of dN_a/dx_i dN_b/dx_j over the unit element (2^dim x 2^dim), by the
    2x2(x2) Gauss rule (exact: the integrands are at most quadratic per direction)."""
    g = [0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)]
    nn = 1 << dim
    L = np.zeros((dim, dim, nn, nn))
    w = 0.5 ** dim
    for p in range(1 << dim):
        xi = [g[(p >> k) & 1] for k in range(dim)]
        G = fem.shape_grad(dim, xi)
        for i in range(dim):
            for j in range(dim):
                L[i, j] += w * np.outer(G[:, i], G[:, j])
    return L


def element_stresses(problem, u):
    """(Nel, d, d) stress tensors at the element centres."""
    p = problem
    dim = p.dim
    B = fem.strain_matrix(dim, fem.shape_grad(dim, [0.5] * dim))
    D0 = fem.constitutive(dim, 1.0, p.nu)
    ed = fem.element_dofs(dim, p.nx, p.ny, p.nz)
    sv = (np.asarray(u)[ed] @ B.T) @ D0.T  # Voigt stresses per unit modulus
    sv = sv * stress_interp(p.rho, p.E0, p.penal)[:, None]
    S = np.zeros((sv.shape[0], dim, dim))
    if dim == 2:
        S[:, 0, 0], S[:, 1, 1] = sv[:, 0], sv[:, 1]
        S[:, 0, 1] = S[:, 1, 0] = sv[:, 2]
    else:
        S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = sv[:, 0], sv[:, 1], sv[:, 2]
        S[:, 1, 2] = S[:, 2, 1] = sv[:, 3]
        S[:, 0, 2] = S[:, 2, 0] = sv[:, 4]
        S[:, 0, 1] = S[:, 1, 0] = sv[:, 5]
    return S


def voigt_pairs(dim):
    """Voigt component v -> the index pairs (i, j) of the stress tensor it fills."""
    if dim == 2:
        return [[(0, 0)], [(1, 1)], [(0, 1), (1, 0)]]
    return [[(0, 0)], [(1, 1)], [(2, 2)], [(1, 2), (2, 1)], [(0, 2), (2, 0)], [(0, 1), (1, 0)]]


def mode_weights(problem, phi):
    """w_e,v = sum over the pairs (i, j) of component v of sum_ab L_ij[a, b] Phi_a . Phi_b,
    (Nel, n_voigt), with Phi masked at fixed DOFs: Phi_e^T K_G,e Phi_e = sum_v sigma_e,v w_e,v."""
    p = problem
    dim = p.dim
    L = gradient_products(dim)
    ed = fem.element_dofs(dim, p.nx, p.ny, p.nz)
    ph = (np.asarray(phi, dtype=np.float64) * fem.free_mask(p.n, p.fixed))[ed]
    ph = ph.reshape(ph.shape[0], 1 << dim, dim)  # (Nel, node a, component)
    G = np.einsum("ijab,eac,ebc->eij", L, ph, ph)
    return np.stack([sum(G[:, i, j] for i, j in pairs) for pairs in voigt_pairs(dim)], axis=1)


def adjoint_rhs(problem, phi):
    """g = d(Phi^T K_sigma(u) Phi)/du = -sum_e E_sigma(rho_e) B^T D_0 w_e (Eq. 7), masked."""
    p = problem
    dim = p.dim
    B = fem.strain_matrix(dim, fem.shape_grad(dim, [0.5] * dim))
    D0 = fem.constitutive(dim, 1.0, p.nu)
    Es = stress_interp(p.rho, p.E0, p.penal)
    ge = -Es[:, None] * (mode_weights(p, phi) @ D0 @ B)  # (Nel, element DOFs)
    g = np.zeros(p.n)
    np.add.at(g, fem.element_dofs(dim, p.nx, p.ny, p.nz), ge)
    return g * fem.free_mask(p.n, p.fixed)


def eigenvalue_sensitivity(problem, u, lam, phi, v):
    """dlambda/drho_e (Eq. 6) for the K-normalised mode phi of eigenvalue lam, the
    displacements u and the adjoint solution v of K v = adjoint_rhs(phi)."""
    p = problem
    dim = p.dim
    m = fem.free_mask(p.n, p.fixed)
    ed = fem.element_dofs(dim, p.nx, p.ny, p.nz)
    rho = np.asarray(p.rho, dtype=np.float64)
    dE = p.penal * rho ** (p.penal - 1.0) * (p.E0 - p.Emin)
    dEs = np.where(rho >= 0.1, p.penal * p.E0 * rho ** (p.penal - 1.0), 0.0)
    B = fem.strain_matrix(dim, fem.shape_grad(dim, [0.5] * dim))
    D0 = fem.constitutive(dim, 1.0, p.nu)
    ue = (np.asarray(u) * m)[ed]
    pe = (np.asarray(phi) * m)[ed]
    ve = (np.asarray(v) * m)[ed]
    Ke = fem.element_stiffness(dim, p.nu)
    s1 = ue @ B.T @ D0.T  # unit-modulus Voigt stresses
    geo = -np.einsum("ev,ev->e", s1, mode_weights(p, phi))  # Phi_e^T K_sigma,e^1 Phi_e
    return (dEs * geo - lam * dE * np.einsum("ea,ab,eb->e", pe, Ke, pe)
            - dE * np.einsum("ea,ab,eb->e", ve, Ke, ue))


def pnorm(lams, p=8):
    """F = (sum_i lambda_i^p)^(1/p) (Eq. 8)."""
    lams = np.asarray(lams, dtype=np.float64)
    return float(np.sum(lams ** p) ** (1.0 / p))


def pnorm_sensitivity(lams, dlams, p=8):
    """dF/drho = F^(1-p) sum_i lambda_i^(p-1) dlambda_i/drho (Eq. 9); dlams (n, Nel)."""
    lams = np.asarray(lams, dtype=np.float64)
    F = pnorm(lams, p)
    return F ** (1.0 - p) * (lams ** (p - 1.0)) @ np.asarray(dlams)


def stress_stiffness(problem, u):
    """K_sigma = -sum_e (sum_ij S_e,ij L_ij) (x) I_d, masked at fixed DOFs, as CSR."""
    p = problem
    dim = p.dim
    L = gradient_products(dim)
    S = element_stresses(p, u)
    H = np.einsum("eij,ijab->eab", S, L)  # (Nel, nn, nn)
    nn = 1 << dim
    nd = dim * nn
    Ke = np.zeros((H.shape[0], nd, nd))
    for c in range(dim):
        Ke[:, c::dim, c::dim] = -H
    ed = fem.element_dofs(dim, p.nx, p.ny, p.nz)
    n = p.n
    rows = np.repeat(ed, nd, axis=1).ravel()
    cols = np.tile(ed, (1, nd)).ravel()
    Ks = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    Ks.sum_duplicates()
    m = fem.free_mask(n, p.fixed)
    Md = sp.diags(m)
    return (Md @ Ks @ Md).tocsr()


def _k_orthonormalize(z, V, KV, K, passes=2):
    """z minus its K-projections on the K-orthonormal columns of V (twice), K-normalised.
    Returns (z, Kz) or (None, None) if z is (numerically) inside span V: its 2-norm dropped
    below 1e-10 of the 2-norm it had."""
    z = np.array(z, dtype=np.float64)
    n0 = np.linalg.norm(z)
    for _ in range(passes):
        if V.shape[1]:
            z = z - V @ (KV.T @ z)
    if not (np.linalg.norm(z) > 1e-10 * n0):
        return None, None
    Kz = K @ z
    nz = np.sqrt(max(z @ Kz, 0.0))
    if not (nz > 0.0):
        return None, None
    return z / nz, Kz / nz


def davidson(Ks, K, M=None, n_eig=6, jmin=10, jmax=25, tol=1e-6, max_iter=1000):
    """Largest eigenpairs of Ks Phi = lambda K Phi by generalized Davidson (Algorithm 2).
    Returns (lambdas descending, Phi (n, n_eig) K-orthonormal, iterations, residuals), the
    iteration count being the number of preconditioner applications.  Convergence of a pair:
    ||Ks q - theta K q|| <= tol ||K q|| |theta| for each of the n_eig largest Ritz pairs."""
    M = (lambda r: r.copy()) if M is None else M
    n = K.shape[0]
    V = np.zeros((n, 0))
    KV = np.zeros((n, 0))
    for k in range(jmin):
        z, Kz = _k_orthonormalize(unit_uniform(n, SALT_GD + k), V, KV, K)
        if z is not None:
            V, KV = np.column_stack([V, z]), np.column_stack([KV, Kz])
    SV = Ks @ V
    it = 0
    while True:
        Hp = V.T @ SV
        Hp = 0.5 * (Hp + Hp.T)
        th, Sv = np.linalg.eigh(Hp)
        order = np.argsort(th)[::-1]
        th, Sv = th[order], Sv[:, order]
        k = min(n_eig, len(th))
        res, conv = [], []
        for i in range(k):
            r = SV @ Sv[:, i] - th[i] * (KV @ Sv[:, i])
            nr = np.linalg.norm(r)
            res.append(nr)
            conv.append(nr <= tol * abs(th[i]) * np.linalg.norm(KV @ Sv[:, i]))
        if all(conv) or it >= max_iter:
            Phi = V @ Sv[:, :k]
            return th[:k], Phi, it, np.array(res)
        t = conv.index(False)
        r = SV @ Sv[:, t] - th[t] * (KV @ Sv[:, t])
        if V.shape[1] >= jmax:
            keep = Sv[:, :jmin]
            V, KV, SV = V @ keep, KV @ keep, SV @ keep
        z, Kz = _k_orthonormalize(M(r), V, KV, K)
        it += 1
        if z is None:
            continue
        V = np.column_stack([V, z])
        KV = np.column_stack([KV, Kz])
        SV = np.column_stack([SV, Ks @ z])
