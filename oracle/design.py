"""Density filter and compliance sensitivities (oracle, FP64, test infrastructure only).

The design variables alpha are mapped to the physical densities by the linear density filter
rho = S alpha (Sec. 2.1, Eq. 1; the filter of Bruns & Tortorelli 2001 with radius 1.5 element
sizes, Sec. 4).  The linear filter weights an element j seen from element e by
w_ej = max(0, r - |c_e - c_j|) (c = element centroids, unit elements, equal volumes) and
normalises every row: S_ej = w_ej / sum_k w_ek.

Compliance sensitivities by the adjoint method (Sec. 2.1, Eq. 3): with the modified SIMP
modulus E(rho) = Emin + (E0 - Emin) rho^p (Eq. 2) and dK/dE_e = the unit-modulus element
matrix Ke placed at element e,
    dF/drho_e = -dE_e/drho_e u_e^T Ke u_e = -p rho_e^(p-1) (E0 - Emin) u_e^T Ke u_e,
and through the filter dF/dalpha = S^T dF/drho.

Parity: pinned (tests/test_oracle_design.py: the closed-form weights of the r = 1.5 stencil,
brute-force filter rows on tiny grids, central finite differences of the compliance f^T u
computed by direct solves, in rho and through the filter in alpha).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


def element_centroids(dim, nx, ny, nz=1):
    """Centroids of the unit elements, element order e = i + nx (j + ny k)."""
    if dim == 2:
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        return np.stack([i.ravel() + 0.5, j.ravel() + 0.5], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([i.ravel() + 0.5, j.ravel() + 0.5, k.ravel() + 0.5], axis=1)


def filter_matrix(dim, nx, ny, nz=1, radius=1.5):
    """S with S_ej = w_ej / sum_k w_ek, w_ej = max(0, radius - |c_e - c_j|), as CSR.  Only
    elements within `radius` contribute, so the neighbourhood is searched over the integer
    offsets |o| <= ceil(radius) along every axis."""
    reach = int(np.ceil(radius))
    nz_ = nz if dim == 3 else 1
    rows, cols, vals = [], [], []
    offs = range(-reach, reach + 1)
    for k in range(nz_):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                rw, cw = [], []
                for oz in (offs if dim == 3 else [0]):
                    for oy in offs:
                        for ox in offs:
                            a, b, c = i + ox, j + oy, k + oz
                            if not (0 <= a < nx and 0 <= b < ny and 0 <= c < nz_):
                                continue
                            w = radius - np.sqrt(ox * ox + oy * oy + oz * oz)
                            if w > 0:
                                rw.append(w)
                                cw.append(a + nx * (b + ny * c))
                tot = sum(rw)
                rows += [e] * len(rw)
                cols += cw
                vals += [w / tot for w in rw]
    n = nx * ny * nz_
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def element_energies(dim, nx, ny, nz, u, nu=0.3):
    """u_e^T Ke u_e for every element (Ke for unit modulus), u: n DOFs."""
    Ke = fem.element_stiffness(dim, nu)
    ed = fem.element_dofs(dim, nx, ny, nz)
    ue = np.asarray(u)[ed]
    return np.einsum("ea,ab,eb->e", ue, Ke, ue)


def compliance_sensitivity(problem, u):
    """dF/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T Ke u_e (Eq. 3), u the displacements."""
    p = problem
    en = element_energies(p.dim, p.nx, p.ny, p.nz, u, p.nu)
    rho = np.asarray(p.rho, dtype=np.float64)
    return -p.penal * rho ** (p.penal - 1.0) * (p.E0 - p.Emin) * en
