"""GPU parity of the steps either side of the solve (Sec. 2.1): the linear density filter, its
transpose and the compliance sensitivities of Eq. 3, called through the C ABI, against the
oracle on the same seeded inputs (FP64: 1e-13 relative)."""
import numpy as np
import pytest

import workloads as W
from oracle import design, fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


@pytest.mark.parametrize("dim,grid", [(2, (1, 1, 1)), (2, (37, 23, 1)), (3, (1, 2, 3)),
                                      (3, (13, 7, 5))])
@pytest.mark.parametrize("radius", [1.5, 1.0, 2.5])
def test_density_filter(lib, ctx, dim, grid, radius):
    p = W.random_problem(dim, *grid, seed=41, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    S = design.filter_matrix(dim, *grid, radius=radius)
    a = np.random.default_rng(2).uniform(0.0, 1.0, p.rho.size)
    for tr, ref in ((False, S @ a), (True, S.T @ a)):
        out = P.density_filter(a, radius=radius, transpose=tr)
        assert np.allclose(out, ref, rtol=1e-13, atol=1e-15)


def test_density_filter_device_path_and_limits(lib, ctx):
    import torch
    p = W.random_problem(2, 20, 10, seed=42, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    a = np.random.default_rng(3).uniform(size=p.rho.size)
    ad = torch.tensor(a, dtype=torch.float64, device="cuda:0")
    od = torch.zeros_like(ad)
    st = lib.load().tomg_density_filter(P.h, 1.5, 0, lib.C.c_void_p(ad.data_ptr()),
                                        lib.C.c_void_p(od.data_ptr()), 1)
    assert st == 0
    assert np.allclose(od.cpu().numpy(), P.density_filter(a), rtol=1e-15, atol=0)
    for bad in (0.0, 3.5):
        with pytest.raises(lib.TomgError):
            P.density_filter(a, radius=bad)


@pytest.mark.parametrize("case", ["mbb", "rand3d"])
def test_compliance_sensitivity(lib, ctx, case):
    p = W.mbb_beam(48, 16) if case == "mbb" else W.random_problem(3, 9, 6, 5, seed=43,
                                                                   contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=2, rtol=1e-10)
    u, res = P.solve(p.f)
    g = P.compliance_sensitivity(u[0])
    ref = design.compliance_sensitivity(p, u[0])
    # rounding scale of each quadratic form: |u_e|^T |Ke| |u_e| (nearly rigid element motions
    # cancel), times the SIMP derivative
    ed = fem.element_dofs(p.dim, p.nx, p.ny, p.nz)
    ue = np.abs(u[0][ed])
    Ka = np.abs(fem.element_stiffness(p.dim, p.nu))
    scale = np.einsum("ea,ab,eb->e", ue, Ka, ue) * p.penal * p.rho ** (p.penal - 1) * (p.E0 - p.Emin)
    assert np.all(np.abs(g - ref) <= 1e-13 * scale + 1e-300)
    # through the filter: dF/dalpha = S^T dF/drho
    S = design.filter_matrix(p.dim, p.nx, p.ny, p.nz, radius=1.5)
    assert np.allclose(P.density_filter(g, transpose=True), S.T @ g, rtol=1e-13,
                       atol=1e-15 * np.abs(g).max())
