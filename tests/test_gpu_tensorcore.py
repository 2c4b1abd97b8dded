"""GPU parity of the hex8 level-0 operator whose element contractions run on the tensor cores
(tcgen05 kind::f16: each element row scaled by a power of two and split into two FP16 parts,
against the exact integer parts of Ke; prec "tc", formerly "tc"), called through the C ABI,
against the CPU oracle on the same seeded inputs.

Tolerance of one apply: 2e-6 per entry of the summed element-product magnitudes
sum_e E_e |Ke| |x_e| (the rounding scale of an element-by-element sum; the assembled |A| |x| is
smaller where element contributions cancel).  The split loses below 2^-22 of each entry (and
2^-36 of the row's largest entry); a CPU emulation of the split on rows spanning eight orders
of magnitude stays within 1.2e-7 of the element scale; the tensor cores' FP32 accumulation adds
a few 2^-24 per term.  Solves: the 1e-8 true relative residual and 1e-6 displacement /
compliance bounds of every other solve test."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, mg, solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return lib.Context(0)


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


# a block owns 31 x 7 nodes in x, y and 8 node layers in z: these grids give one and several
# blocks per axis, ragged last blocks, and single-element extents
GRIDS = [(1, 1, 1), (3, 2, 1), (9, 8, 7), (13, 7, 5), (30, 6, 7), (31, 7, 8), (40, 9, 6),
         (62, 14, 17), (65, 20, 9)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("contrast", ["minmax", "threshold"])
def test_tc_operator_apply(lib, ctx, grid, contrast):
    p = W.random_problem(3, *grid, seed=31, contrast=contrast)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="jacobi", prec="tc")
    A0 = mg.fine_operator(p)
    E = fem.simp(p.rho, p.E0, p.Emin, p.penal)
    Kabs = fem.masked_operator(abs(fem.assemble(3, p.nx, p.ny, p.nz, E,
                                                np.abs(fem.element_stiffness(3, p.nu)))), p.fixed)
    rng = np.random.default_rng(7)
    for x in (rng.standard_normal(p.n), rng.standard_normal(p.n) * 10.0 ** rng.uniform(-4, 4, p.n)):
        y = P.level_apply(0, x, "tc")
        scale = Kabs @ np.abs(x)
        assert np.all(np.abs(y - A0 @ x) <= 2e-6 * scale + 1e-300)


@pytest.mark.parametrize("grid", [(13, 7, 5), (62, 14, 17)])
def test_tc_matches_cuda_core_fp32(lib, ctx, grid):
    """Both FP32 level-0 kernels compute the same masked operator; they differ only in rounding."""
    p = W.random_problem(3, *grid, seed=32, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="jacobi", prec="fp32")
    x = np.random.default_rng(3).standard_normal(p.n)
    y32 = P.level_apply(0, x, "fp32")
    ytc = P.level_apply(0, x, "tc")
    y64 = P.level_apply(0, x, "fp64")
    assert relerr(ytc, y64) < 1e-6
    assert relerr(y32, y64) < 1e-6
    # fixed DOFs pass x through unchanged in every kernel
    fixed = np.asarray(p.fixed)
    assert np.array_equal(ytc[fixed], y32[fixed])


def test_tc_vcycle_close_to_fp32(lib, ctx):
    p = W.random_problem(3, 24, 12, 10, seed=33, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    r = np.random.default_rng(4).standard_normal(p.n) * fem.free_mask(p.n, p.fixed)
    P.setup(pc="gmg", n_levels=3, prec="fp64")
    z64 = P.vcycle(r)
    P.setup(pc="gmg", n_levels=3, prec="tc")
    ztc = P.vcycle(r)
    P.setup(pc="gmg", n_levels=3, prec="fp32")
    z32 = P.vcycle(r)
    assert relerr(ztc, z64) < 1e-4
    assert relerr(ztc, z32) < 1e-4


@pytest.mark.parametrize("pc,kw", [("gmg", dict(n_levels=3)),
                                   ("hybrid", dict(n_geo_levels=2, max_coarse_dofs=200))])
def test_tc_solve_vs_direct(lib, ctx, pc, kw):
    p = W.cantilever_3d(16, 8, 8, seed=0, sigma=2.0)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc=pc, prec="tc", rtol=1e-8, **kw)
    u, res = P.solve(p.f)
    r = res[0]
    assert r["status"] == 0, r
    ref = osolve.direct(p)
    A0 = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * p.f[0]
    assert np.linalg.norm(b - A0 @ u[0]) / np.linalg.norm(b) <= 1.05e-8
    assert relerr(u, ref["u"]) <= 1e-6
    assert abs(r["compliance"] - ref["compliance"][0]) <= 1e-6 * abs(ref["compliance"][0])
    # the FP32 CUDA-core V-cycle needs the same number of outer iterations up to rounding drift
    P.setup(pc=pc, prec="fp32", rtol=1e-8, **kw)
    _, res32 = P.solve(p.f)
    assert abs(res32[0]["iterations"] - r["iterations"]) <= 2


def test_tc_multi_rhs_concurrent_slots(lib, ctx):
    """Several right-hand sides on concurrent solve slots share the tensor-core kernel; each result
    equals its solve alone (fixed-order sums in the kernel: bit-identical)."""
    p = W.random_problem(3, 20, 10, 10, seed=34, contrast="minmax", nrhs=3)
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=3, prec="tc", concurrency=3)
    U, res = P.solve(p.f)
    for j in range(3):
        assert res[j]["status"] == 0
        u1, _ = P.solve(p.f[j])
        assert np.array_equal(U[j], np.asarray(u1).reshape(-1))


def test_tc_wait_timeout_path(lib, ctx):
    """The bounded-wait path of the tensor-core kernel, exercised without a fault: with the test
    hook set (tomg_debug_tc_wait_limit) the blocks' waits watch a barrier that nothing arrives
    on and give up after one poll, so every block records the failure, waits with the full limit
    for the MMAs it has in flight, frees its tensor memory and returns; the apply reports
    TOMG_E_TIMEOUT.  With the hook cleared the record is clear and the operator and a solve give
    the results of before."""
    p = W.random_problem(3, 40, 20, 18, seed=35, contrast="minmax")
    P = lib.Problem.from_workload(ctx, p)
    P.setup(pc="gmg", n_levels=3, prec="tc", rtol=1e-8)
    x = np.random.default_rng(8).standard_normal(p.n)
    y_ref = P.level_apply(0, x, "tc")
    u_ref, r_ref = P.solve(p.f)
    timeouts = 0
    lib.debug_tc_wait_limit(1)
    try:
        for _ in range(3):
            try:
                P.level_apply(0, x, "tc")
            except lib.TomgError as e:
                assert e.status == lib.E_TIMEOUT, e
                timeouts += 1
    finally:
        lib.debug_tc_wait_limit(0)
    assert timeouts == 3
    assert np.array_equal(P.level_apply(0, x, "tc"), y_ref)
    P.setup(pc="gmg", n_levels=3, prec="tc", rtol=1e-8)
    u, r = P.solve(p.f)
    assert r[0]["status"] == 0 and r[0]["iterations"] == r_ref[0]["iterations"]
    assert np.array_equal(u, u_ref)
