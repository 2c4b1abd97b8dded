"""Pins for oracle.design: the linear density filter and the compliance sensitivities."""
import numpy as np
import pytest

import workloads as W
from oracle import design, fem


def test_filter_weights_closed_form():
    """r = 1.5 on unit elements: weights 1.5 (self), 0.5 (face neighbours), 1.5 - sqrt(2)
    (diagonal neighbours in a plane), 0 beyond; an interior row of the 2D filter therefore
    sums 1.5 + 4 * 0.5 + 4 * (1.5 - sqrt 2) before normalisation."""
    S = design.filter_matrix(2, 5, 5, radius=1.5).toarray()
    e = 2 + 5 * 2  # interior element
    tot = 1.5 + 4 * 0.5 + 4 * (1.5 - np.sqrt(2.0))
    assert S[e, e] == pytest.approx(1.5 / tot, rel=1e-15)
    assert S[e, e + 1] == pytest.approx(0.5 / tot, rel=1e-15)
    assert S[e, e + 6] == pytest.approx((1.5 - np.sqrt(2.0)) / tot, rel=1e-15)
    assert S[e, e + 2] == 0.0 and np.count_nonzero(S[e]) == 9
    # 3D interior row: 1 + 6 face + 12 edge neighbours (corners at sqrt 3 > 1.5 drop out)
    S3 = design.filter_matrix(3, 5, 5, 5, radius=1.5).toarray()
    e3 = 2 + 5 * (2 + 5 * 2)
    assert np.count_nonzero(S3[e3]) == 19


@pytest.mark.parametrize("dim,grid", [(2, (4, 3, 1)), (3, (3, 3, 2))])
@pytest.mark.parametrize("radius", [1.5, 2.2])
def test_filter_rows_brute_force(dim, grid, radius):
    """Every row against the definition evaluated over all element pairs."""
    S = design.filter_matrix(dim, *grid, radius=radius).toarray()
    c = design.element_centroids(dim, *grid)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
    w = np.maximum(0.0, radius - d)
    ref = w / w.sum(axis=1, keepdims=True)
    assert np.allclose(S, ref, rtol=1e-14, atol=0)
    assert np.allclose(S.sum(axis=1), 1.0, rtol=1e-14)  # a uniform field passes unchanged


def _compliance(p, rho):
    q = W.Problem(p.name, p.dim, p.nx, p.ny, p.nz, rho, p.fixed, p.f, E0=p.E0, Emin=p.Emin,
                  penal=p.penal, nu=p.nu)
    K = fem.stiffness(q)
    u = fem.direct_solve(K, q.fixed, q.f)
    return fem.compliance(q.f, u)[0], u[0]


@pytest.mark.parametrize("dim,grid", [(2, (6, 4, 1)), (3, (3, 2, 2))])
def test_sensitivity_matches_finite_differences(dim, grid):
    """dF/drho_e (Eq. 3) against central differences of F = f^T u with direct solves."""
    p = W.random_problem(dim, *grid, seed=4, contrast="minmax")
    c0, u = _compliance(p, p.rho)
    g = design.compliance_sensitivity(p, u)
    for e in range(0, p.rho.size, max(1, p.rho.size // 7)):
        # step relative to rho_e: truncation O((h / rho)^2) ~ 1e-6; much smaller steps drown
        # in the rounding of the solves (F ~ 3e3)
        h = 1e-3 * p.rho[e]
        rp, rm = p.rho.copy(), p.rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (_compliance(p, rp)[0] - _compliance(p, rm)[0]) / (2 * h)
        # near rho = 1e-3 the difference quotient itself is only good to a few 1e-4
        tol = 1e-4 if p.rho[e] >= 0.05 else 1e-3
        assert g[e] == pytest.approx(fd, rel=tol, abs=1e-7 * abs(c0))
    assert np.all(g <= 0.0)  # more material never increases the compliance


def test_filtered_sensitivity_chain_rule():
    """dF/dalpha = S^T dF/drho against central differences in alpha through rho = S alpha."""
    p = W.random_problem(2, 6, 4, seed=5, contrast="minmax")
    S = design.filter_matrix(2, p.nx, p.ny, radius=1.5)
    alpha = np.clip(p.rho, 0.05, 1.0)
    rho = S @ alpha
    q = W.Problem(p.name, 2, p.nx, p.ny, 1, rho, p.fixed, p.f, E0=p.E0, Emin=p.Emin,
                  penal=p.penal, nu=p.nu)
    _, u = _compliance(q, rho)
    ga = S.T @ design.compliance_sensitivity(q, u)
    h = 1e-4  # alpha >= 0.05
    for j in (0, 5, 11, 23):
        ap, am = alpha.copy(), alpha.copy()
        ap[j] += h
        am[j] -= h
        fd = (_compliance(q, S @ ap)[0] - _compliance(q, S @ am)[0]) / (2 * h)
        assert ga[j] == pytest.approx(fd, rel=1e-4)
