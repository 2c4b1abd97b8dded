"""The allocation-free operator apply (tomg_fine_apply_f32_noalloc) gives the same result as the
regular FP32 apply (tomg_level_apply on level 0), on two calls in a row, through the C ABI.

It exists for callers that may not allocate device memory where they apply the operator (their
device memory belongs to another allocator, or they cannot pay the device-wide synchronisation
that freeing memory implies).  This file is named so that pytest collects it last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _problem(lib, ctx, p):
    P = lib.Problem(ctx, p.dim, p.nx, p.ny, p.nz, p.E0, p.Emin, p.penal, p.nu)
    P.set_fixed_dofs(p.fixed)
    P.set_density(p.rho)
    return P


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_noalloc_matches_regular_apply_twice(lib, case):
    import torch
    stream = torch.cuda.current_stream()
    ctx = lib.Context(0, stream)
    if case == "2d":
        p = W.random_problem(2, 203, 101, seed=21, contrast="threshold")
    else:
        p = W.random_problem(3, 37, 19, 11, seed=22, contrast="minmax")
    P = _problem(lib, ctx, p)
    P.setup(pc="jacobi")  # the regular apply needs a setup; the allocation-free one does not
    rng = np.random.default_rng(5)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(p.n), dtype=torch.float64, device="cuda:0")
        y_ref = P.level_apply(0, x, "fp32")
        y = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda:0")
        P.fine_apply_f32_noalloc(x, y)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), call
        assert np.array_equal(got, ref), call  # same kernels, same inputs: bit-identical


def test_noalloc_rejects_oversized_problem(lib):
    ctx = lib.Context(0)
    P = lib.Problem(ctx, 2, 800, 700)  # 2 x 801 x 701 = 1,123,002 DOFs > 1,048,576
    assert P.n == 2 * 801 * 701 and P.n > 1 << 20
    P.set_density(np.ones(800 * 700))
    import torch
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda:0")
    y = torch.zeros_like(x)
    with pytest.raises(lib.TomgError) as e:
        P.fine_apply_f32_noalloc(x, y)
    assert e.value.status == lib.E_INVALID
    assert "at most" in str(e.value)
