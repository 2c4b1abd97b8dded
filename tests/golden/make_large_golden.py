"""Writes the oracle reference values of the benchmark workloads to text fixtures in this
folder: the 3D cantilever 192x96x96 and the 16 right-hand sides of the batched 128x64x64 case
(solved by PCG, see below), and the 2D cantilever 768x384 and the MBB beam 96x32 (solved by the
oracle's refined sparse direct solve).

The 3D workloads are too large for a sparse direct solve on a host.  The method reaches the unique
solution of K(rho) u = f with u = 0 on fixed DOFs (Sec. 3.1), so the oracle computes that
solution by textbook PCG (oracle.krylov.pcg) on the assembled masked CSR operator, with the
oracle's own hybrid multigrid V-cycle (FP64 throughout) as preconditioner, iterating to a
relative residual of 1e-12 or until the FP64 residual stops decreasing.  The true residual is
recomputed from the assembled operator.  As an independent check of the accuracy reached,
right-hand side 0 of every workload is solved a second time with a different preconditioner
(the oracle's geometric V-cycle with one point-block Jacobi sweep) and the relative
difference of the two solutions is recorded.

Each fixture holds, per right-hand side:
  * the compliance f^T u (Eq. 1), ||u||_2, ||u||_inf, the iteration count, the true residual;
  * u . g_i for 8 seeded N(0,1) vectors g_i (numpy default_rng(1000 + i), length n), whose
    differences estimate ||u - u_ref||_2 on the whole vector;
  * u at 200 seeded uniformly drawn DOFs (default_rng(2000 + rhs)), at the DOF of largest
    |u| and at the (at most 16 most) loaded DOFs.

Run from the repository root (about an hour and 20 GB of host memory):
    python tests/golden/make_large_golden.py [cantilever3d] [batched3d] [cantilever2d] [mbb]
It imports only ``oracle``, ``workloads`` and the fixture reader ``refs`` beside it (for the
seeded probe vectors).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

sys.path.insert(0, HERE)

import workloads as W  # noqa: E402
from oracle import fem, krylov, mg, solve as osolve  # noqa: E402
from refs import projections  # noqa: E402

N_SAMPLE = 200


def sample_dofs(u, f, free, rhs):
    rng = np.random.default_rng(2000 + rhs)
    uni = np.sort(rng.choice(np.flatnonzero(free), size=N_SAMPLE, replace=False))
    loaded = np.argsort(-np.abs(f))[:16]
    loaded = loaded[np.abs(f[loaded]) > 0]
    extra = np.unique(np.concatenate([[int(np.argmax(np.abs(u)))], loaded]))
    return uni, extra


def solve_to_floor(A0, b, M, rtol=1e-12, max_iter=600):
    """PCG to rtol; PCG's recursive residual keeps decreasing below the FP64 floor of the true
    residual, so the run is also capped at max_iter."""
    t0 = time.perf_counter()
    x, it, hist = krylov.pcg(A0, b, M=M, rtol=rtol, max_iter=max_iter)
    nb = np.linalg.norm(b)
    true = np.linalg.norm(b - A0 @ x) / nb
    return x, it, true, time.perf_counter() - t0


def run(p, name, n_geo, cap, out_path):
    t0 = time.perf_counter()
    A0 = mg.fine_operator(p)
    print("%s: fine operator %.1f s, nnz %d" % (name, time.perf_counter() - t0, A0.nnz), flush=True)
    t1 = time.perf_counter()
    H = osolve.build(p, pc="hybrid", n_geo=n_geo, cap=cap, A0=A0, smoother="chebyshev")
    print("%s: hybrid hierarchy %.1f s, levels %s" % (name, time.perf_counter() - t1,
                                                       [A.shape[0] for A in H.A]), flush=True)
    free = fem.free_mask(p.n, p.fixed)
    G = projections(p.n)
    lines = []
    lines.append("# oracle reference of %s: %d DOFs, %d right-hand sides" % (name, p.n, p.nrhs))
    lines.append("# PCG (FP64) with the oracle's hybrid V-cycle (%d geometric levels, SA-AMG "
                 "below %d DOFs, degree-2 Chebyshev), rtol 1e-12 or 600 iterations" % (n_geo, cap))
    lines.append("# written by tests/golden/make_large_golden.py (oracle only)")
    for r in range(p.nrhs):
        b = free * p.f[r]
        u, it, true, secs = solve_to_floor(A0, b, lambda v: mg.vcycle(H, v))
        print("%s rhs %d: %d iterations, true residual %.3e, %.0f s" % (name, r, it, true, secs),
              flush=True)
        comp = float(p.f[r] @ u)
        lines.append("rhs %d n %d iterations %d true_rel_residual %.6e" % (r, p.n, it, true))
        lines.append("compliance %.17e" % comp)
        lines.append("norm2 %.17e" % np.linalg.norm(u))
        lines.append("norminf %.17e" % np.abs(u).max())
        lines.append("proj " + " ".join("%.17e" % (g @ u) for g in G))
        if r == 0:
            Hg = osolve.build(p, pc="gmg", n_levels=n_geo + 2, A0=A0, smoother="jacobi")
            u2, it2, true2, secs2 = solve_to_floor(A0, b, lambda v: mg.vcycle(Hg, v))
            d = np.linalg.norm(u - u2) / np.linalg.norm(u)
            dc = abs(float(p.f[r] @ u2) - comp) / abs(comp)
            print("%s rhs 0 cross-check: %d iterations, true residual %.3e, rel diff %.3e, "
                  "compliance diff %.3e, %.0f s" % (name, it2, true2, d, dc, secs2), flush=True)
            lines.append("crosscheck gmg_jacobi iterations %d true_rel_residual %.6e "
                         "rel_u_diff %.6e rel_compliance_diff %.6e" % (it2, true2, d, dc))
            del Hg, u2
        uni, extra = sample_dofs(u, p.f[r], free.astype(bool), r)
        lines.append("uniform %d" % len(uni))
        lines += ["%d %.17e" % (i, u[i]) for i in uni]
        lines.append("extra %d" % len(extra))
        lines += ["%d %.17e" % (i, u[i]) for i in extra]
    with open(out_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", out_path, flush=True)


def run_direct(p, name, out_path):
    """Reference of a 2D workload: the oracle's sparse LU with iterative refinement."""
    t0 = time.perf_counter()
    ref = osolve.direct(p)
    A0 = mg.fine_operator(p)
    free = fem.free_mask(p.n, p.fixed)
    G = projections(p.n)
    print("%s: direct solve %.1f s" % (name, time.perf_counter() - t0), flush=True)
    lines = ["# oracle reference of %s: %d DOFs, %d right-hand sides" % (name, p.n, p.nrhs),
             "# sparse LU of the reduced system with iterative refinement (oracle.solve.direct)",
             "# written by tests/golden/make_large_golden.py (oracle only)"]
    U = np.atleast_2d(ref["u"])
    for r in range(p.nrhs):
        u = U[r]
        b = free * p.f[r]
        true = np.linalg.norm(b - A0 @ u) / np.linalg.norm(b)
        lines.append("rhs %d n %d iterations 0 true_rel_residual %.6e" % (r, p.n, true))
        lines.append("compliance %.17e" % float(p.f[r] @ u))
        lines.append("norm2 %.17e" % np.linalg.norm(u))
        lines.append("norminf %.17e" % np.abs(u).max())
        lines.append("proj " + " ".join("%.17e" % (g @ u) for g in G))
        uni, extra = sample_dofs(u, p.f[r], free.astype(bool), r)
        lines.append("uniform %d" % len(uni))
        lines += ["%d %.17e" % (i, u[i]) for i in uni]
        lines.append("extra %d" % len(extra))
        lines += ["%d %.17e" % (i, u[i]) for i in extra]
    with open(out_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", out_path, flush=True)


def main():
    which = sys.argv[1:] or ["cantilever3d", "batched3d", "cantilever2d", "mbb"]
    if "mbb" in which:
        run_direct(W.mbb_beam(96, 32), "mbb_96x32", os.path.join(HERE, "mbb_96x32.txt"))
    if "cantilever2d" in which:
        run_direct(W.cantilever_2d(768, 384, seed=0), "cantilever2d_768x384",
                   os.path.join(HERE, "cantilever2d_768x384.txt"))
    if "cantilever3d" in which:
        run(W.cantilever_3d(192, 96, 96, seed=0), "cantilever3d_192x96x96", 3, 1000,
            os.path.join(HERE, "cantilever3d_192x96x96.txt"))
    if "batched3d" in which:
        run(W.batched_3d(), "batched3d_128x64x64_x16", 3, 1000,
            os.path.join(HERE, "batched3d_128x64x64.txt"))


if __name__ == "__main__":
    main()
