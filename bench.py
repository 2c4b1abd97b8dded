"""Throughput of the multigrid-preconditioned CG solve of the SIMP elasticity system.

One step = one whole pass of the hot path on the 3D cantilever (192 x 96 x 96 hex8 elements,
5,447,811 DOFs, seeded smoothed density in [1e-3, 1] with p = 3, face x = 0 clamped, line load
on the far bottom edge): SIMP moduli from the density already resident in HBM, preconditioner
setup (two geometric Galerkin coarsenings, smoothed aggregation below to < 1000 DOFs, smoother
bounds, coarse Cholesky) and a solve to a true relative residual of 1e-8.  Headline: mixed
precision (FP32 V-cycle with tensor-core element contractions inside FP64 flexible CG);
the FP64 V-cycle PCG is measured beside it.  Every result is compared with the oracle's
reference solution (tests/golden).  The other workloads (MBB beam, 2D cantilever with GMG /
AMG / hybrid, the 16 right-hand sides of the batched 3D case, the serving stream) are
reported under their own keys.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  The reference arm times the CPU oracle (plain FP64 numpy /
scipy PCG with the same kind of hierarchy): complete solves of the same cantilever at 1/27 of
the elements, scaled by the DOF ratio.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))

METRIC = "MG-PCG solves/sec & DOF-iters/sec @1e-8 residual, mixed vs FP64; p50/p99 latency"
WORKLOAD = dict(nx=192, ny=96, nz=96, seed=0)
REF_NAME = "cantilever3d_192x96x96"
HEADLINE = dict(pc="hybrid", n_geo_levels=3, max_coarse_dofs=1000, rtol=1e-8, max_iter=2000)
HEAD_PREC = "tc"
# the oracle's complete solves run on the same cantilever with 1/27 of the elements
SAMPLE_GRID = (64, 32, 32)


def smoother_label(args):
    if args.smoother == "chebyshev":
        return "chebyshev degree %d" % args.cheb_degree
    if args.smoother == "gmres":
        return "gmres 2 steps per smoothing"
    return args.smoother


def workload_label():
    return ("3D cantilever hex8 %dx%dx%d (5,447,811 DOFs), seeded smoothed density in [1e-3, 1], "
            "p = 3, face x = 0 clamped, line load on the far bottom edge"
            % (WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["nz"]))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tomg")
    ap.add_argument("--graph-mode", type=int, default=2,
                    help="2: whole solve in one graph (device while loop); 1: one graph per "
                         "iteration (host polls); 0: no graphs")
    ap.add_argument("--smoother", default="chebyshev", choices=["jacobi", "chebyshev", "gmres"],
                    help="V-cycle smoother of the timed solves; the paper's runs use one Jacobi "
                         "sweep, which is measured beside the headline as `jacobi`")
    ap.add_argument("--cheb-degree", type=int, default=2)
    ap.add_argument("--serving", type=int, default=256,
                    help="clients of the mixed-size serving stream (0: skip)")
    ap.add_argument("--serving-updates", type=int, default=10)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--batched", type=int, default=1,
                    help="also time the 16 right-hand sides of the 3D 128x64x64 case (0: skip)")
    ap.add_argument("--others", type=int, default=1,
                    help="also time the MBB beam and the 2D cantilever (0: skip)")
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the solver variants (GMRES smoother, FGMRES, design "
                         "iterations, stability) on the 2D workloads (0: skip)")
    ap.add_argument("--kernel", default=None, choices=["outer", "residual", "jacobi", "apply"],
                    help="time one level-0 operator kernel alone (for profiler captures) instead "
                         "of the solve: outer = FP64 q = K p with its dot, the others the "
                         "V-cycle's kernels in --kernel-prec")
    ap.add_argument("--kernel-prec", default="fp32")
    ap.add_argument("--kernel-grid", default="2048x1024",
                    help="element counts of the cantilever used by --kernel (NXxNY or NXxNYxNZ)")
    ap.add_argument("--kernel-reps", type=int, default=20)
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the comparison variants (FP64 V-cycle, the paper's Jacobi sweep)")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 3 + i and r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """Largest per-rank value (the slowest rank's time) across the process group."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: int, world: int, total_ms: float) -> float:
    """Whole-job rate: the units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1e3)


T_START = time.perf_counter()


def progress(what):
    """One line per phase on stderr (the JSON line alone goes to stdout)."""
    print("[bench %7.1f s] %s" % (time.perf_counter() - T_START, what), file=sys.stderr,
          flush=True)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


def accuracy_of(u, res, ref, G):
    """Error of one result against the oracle reference (tests/golden/refs.py)."""
    import refs
    a = refs.accuracy(np.asarray(u), res["compliance"], ref, G)
    a["rel_residual"] = res["rel_residual"]
    return {k: float("%.3e" % v) for k, v in a.items()}


def worst(accs):
    return {k: max(a[k] for a in accs) for k in accs[0]}


class Stepper:
    """One problem with its density and load resident on the device; step() = moduli + setup +
    solve from u = 0, timed with CUDA events on the context stream (L2 flushed first)."""

    def __init__(self, tomg, ctx, p, stream, dev):
        import torch
        self.torch, self.ctx, self.p, self.stream = torch, ctx, p, stream
        self.P = tomg.Problem.from_workload(ctx, p)
        self.rho_d = torch.tensor(p.rho, dtype=torch.float64, device=dev)
        self.f_d = torch.tensor(p.f[0], dtype=torch.float64, device=dev)
        self.u_d = torch.zeros_like(self.f_d)
        self.u_last = self.u_d
        self.flush = torch.empty(256 << 20, dtype=torch.int8, device=dev)  # > 129 MB L2

    def step(self, prec, opts):
        self.u_d.zero_()
        self.P.set_density(self.rho_d)
        self.P.setup(prec=prec, **opts)
        self.u_last, res = self.P.solve(self.f_d, u0=self.u_d)
        return res[0]

    def timed(self, prec, opts, K, Wm, world=1):
        torch = self.torch
        for _ in range(Wm):
            self.step(prec, opts)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times, results = [], []
        l0 = self.ctx.kernel_launches()
        for _ in range(K):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            r = self.step(prec, opts)
            e1.record(self.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            results.append(r)
        launches = self.ctx.kernel_launches() - l0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return times, results, launches

    def summary(self, times, results):
        its = [r["iterations"] for r in results]
        return {"solves_per_s": len(times) / (sum(times) / 1e3),
                "dof_iters_per_s": self.p.n * sum(its) / (sum(times) / 1e3),
                "iterations": statistics.median(its),
                "latency_ms": {"p50": float(np.percentile(times, 50)),
                               "p99": float(np.percentile(times, 99))},
                "setup_ms": statistics.median(r["setup_ms"] for r in results),
                "solve_ms": statistics.median(r["solve_ms"] for r in results),
                "rel_residual_max": max(r["rel_residual"] for r in results),
                "failed_steps": sum(1 for r in results
                                    if r["status"] != 0 or r["rel_residual"] > 1e-8)}


def run_gpu(args, rank, world, local):
    import torch
    import refs
    import workloads as W
    from paper_2001_01655_gb300 import tomg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    ctx = tomg.Context(local, stream)
    p = W.cantilever_3d(**WORKLOAD)
    S = Stepper(tomg, ctx, p, stream, dev)
    opts = dict(HEADLINE, use_graph=args.graph_mode, smoother=args.smoother,
                cheb_degree=args.cheb_degree)
    ref = refs.load(REF_NAME)[0]
    G = refs.projections(p.n)

    progress("headline")
    with Clocks(local) as clk:
        times, results, launches = S.timed(HEAD_PREC, opts, args.steps, args.warmup, world)
    total_ms = max_over_ranks(sum(times), world, device=dev)
    head = S.summary(times, results)
    out = {
        "metric": METRIC,
        "value": throughput(args.steps, world, total_ms),
        "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 outer / f32 V-cycle (tensor-core element contractions)",
        "data": "synthetic",
        "config": {"workload": workload_label(),
                   "preconditioner": "hybrid: 3 geometric levels, SA-AMG below to < 1000 DOFs",
                   "rtol": 1e-8, "smoother": smoother_label(args),
                   "step": "SIMP moduli + hierarchy setup + FCG solve from u = 0",
                   "l2": "flushed between timed steps (256 MB write); vectors 44 MB each",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "dof_iters_per_s": world * head["dof_iters_per_s"],
        "iterations": head["iterations"],
        "latency_ms": head["latency_ms"],
        "setup_ms": head["setup_ms"], "solve_ms": head["solve_ms"],
        "rel_residual_max": head["rel_residual_max"],
        "failed_steps": head["failed_steps"],
        "accuracy": accuracy_of(S.u_last.cpu().numpy(), results[-1], ref, G),
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    progress("fp64 + jacobi variants")
    if not args.no_fp64:
        t64, r64, _ = S.timed("fp64", opts, max(3, args.steps // 2), 1)
        out["fp64"] = dict(S.summary(t64, r64),
                           accuracy=accuracy_of(S.u_last.cpu().numpy(), r64[-1], ref, G))
        out["mixed_over_fp64"] = out["value"] / out["fp64"]["solves_per_s"]
        if args.smoother != "jacobi":
            # the paper's smoother (one weighted point-block Jacobi sweep), mixed and FP64
            oj = dict(opts, smoother="jacobi")
            jac = {}
            for prec, key in ((HEAD_PREC, "mixed"), ("fp64", "fp64")):
                tj, rj, _ = S.timed(prec, oj, max(3, args.steps // 4), 1)
                jac[key] = dict(S.summary(tj, rj),
                                accuracy=accuracy_of(S.u_last.cpu().numpy(), rj[-1], ref, G))
            out["jacobi"] = jac
    progress("e2e")
    # end to end through the C ABI with host buffers in pinned memory: density, load and the
    # initial guess copied in, u copied out, inside the timed region
    rho_h = torch.tensor(p.rho, dtype=torch.float64).pin_memory()
    f_h = torch.tensor(p.f[0], dtype=torch.float64).pin_memory()
    u_h = torch.zeros_like(f_h).pin_memory()
    e2e = []
    for k in range(max(3, args.steps // 4) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u_h.zero_()
        S.P.set_density(rho_h)
        S.P.setup(prec=HEAD_PREC, **opts)
        _, res = S.P.solve(f_h, out=u_h)
        if k:
            e2e.append(time.perf_counter() - t0)
    out["e2e"] = {"value": world / statistics.median(e2e), "unit": "solves/s",
                  "h2d_bytes_per_step": int(8 * (rho_h.numel() + 2 * f_h.numel())),
                  "d2h_bytes_per_step": int(8 * f_h.numel()),
                  "host_buffers": "pinned",
                  "accuracy": accuracy_of(u_h.numpy(), res[0], ref, G)}
    progress("roofline")
    out["roofline"] = roofline(S.P, p, head, opts)
    progress("mbb + 2D cantilever")
    if args.others:
        out["mbb_96x32"] = mbb_run(tomg, ctx, stream, dev, args)
        out["cantilever2d_768x384"] = cantilever2d_run(tomg, ctx, stream, dev, args)
    progress("batched")
    if args.batched:
        out["batched"] = batched_run(tomg, ctx, args.slots, smoother=args.smoother,
                                     cheb_degree=args.cheb_degree)
    progress("serving")
    if args.serving > 0:
        out["serving"] = serving_run(tomg, ctx, args.serving, args.serving_updates, args.slots)
    progress("variants")
    if args.variants and not args.no_fp64:
        out["variants_2d"] = variants_run(tomg, ctx, stream, dev, args)
    return out


def mbb_run(tomg, ctx, stream, dev, args):
    """The MBB beam as configured: FP64 GMG-PCG with 4 levels (130 coarse DOFs) and one
    point-block Jacobi sweep, rel. residual 1e-8."""
    import refs
    import workloads as W
    p = W.mbb_beam(96, 32)
    S = Stepper(tomg, ctx, p, stream, dev)
    o = dict(pc="gmg", n_levels=4, smoother="jacobi", rtol=1e-8, use_graph=args.graph_mode)
    t, r, _ = S.timed("fp64", o, 20, 3)
    ref = refs.load("mbb_96x32")[0]
    return dict(S.summary(t, r), workload="MBB beam quad4 96x32 (6,402 DOFs), rho = 0.5",
                preconditioner="GMG 4 levels, FP64 PCG, Jacobi",
                accuracy=accuracy_of(S.u_last.cpu().numpy(), r[-1], ref,
                                     refs.projections(p.n)))


def cantilever2d_run(tomg, ctx, stream, dev, args):
    """The 2D cantilever (768 x 384 quad4, thin 0/1 members, 1e9 contrast) with the paper's three
    hierarchies (Sec. 4.1-4.3): GMG to < 1500 DOFs (6 levels), SA-AMG to < 1500 DOFs, and the
    hybrid (one geometric coarsening, then SA-AMG); mixed precision and FP64 each."""
    import refs
    import workloads as W
    p = W.cantilever_2d(768, 384, seed=0)
    S = Stepper(tomg, ctx, p, stream, dev)
    ref = refs.load("cantilever2d_768x384")[0]
    G = refs.projections(p.n)
    out = {"workload": "2D cantilever quad4 768x384 (592,130 DOFs), seeded thin 0/1 members "
                       "(1e9 contrast), left edge clamped, unit load right mid-edge",
           "smoother": smoother_label(args)}
    for pc in ("hybrid", "gmg", "amg"):
        o = dict(pc=pc, max_coarse_dofs=1500, n_geo_levels=2, rtol=1e-8, max_iter=2000,
                 use_graph=args.graph_mode, smoother=args.smoother, cheb_degree=args.cheb_degree)
        res = {"levels": None}
        for prec, key in (("fp32", "mixed"), ("fp64", "fp64")):
            t, r, _ = S.timed(prec, o, 10 if pc != "gmg" else 2, 3 if pc != "gmg" else 1)
            res[key] = dict(S.summary(t, r), converged=all(x["status"] == 0 for x in r),
                            accuracy=accuracy_of(S.u_last.cpu().numpy(), r[-1],
                                                                   ref, G))
        res["levels"] = [S.P.level_info(l)["n_dofs"] for l in range(S.P.num_levels())]
        out[pc] = res
    return out


def variants_run(tomg, ctx, stream, dev, args):
    """The solver variants the paper studies beside the headline, on the 2D cantilever: the
    GMRES smoother (Sec. 4.1), flexible GMRES(30) as the outer solver, design iterations around
    the solve (Sec. 2.1), and the stability chain on the paper's 2D column (Sec. 2.2, 4.2)."""
    import workloads as W
    p = W.cantilever_2d(768, 384, seed=0)
    S = Stepper(tomg, ctx, p, stream, dev)
    opts = dict(pc="hybrid", max_coarse_dofs=1500, n_geo_levels=2, rtol=1e-8, max_iter=2000,
                use_graph=args.graph_mode, smoother="chebyshev", cheb_degree=2)
    gm = {}
    for steps_ in (2, 4):
        og = dict(opts, smoother="gmres", gmres_steps=steps_)
        tg, rg, _ = S.timed("fp32", og, 3, 1)
        gm["steps_%d" % steps_] = {
            "solves_per_s": len(tg) / (sum(tg) / 1e3),
            "iterations": statistics.median(r["iterations"] for r in rg),
            "rel_residual_max": max(r["rel_residual"] for r in rg)}
    return {"workload": "2D cantilever quad4 768x384 (variants); 2D column 256x1024 (stability)",
            "gmres_smoother": gm,
            "fgmres": fgmres_run(S.P, opts, S.rho_d, S.f_d, S.u_d),
            "design_iteration": design_run(S.P, opts, p, S.rho_d, S.f_d),
            "stability": stability_run(tomg, ctx, opts)}


def fgmres_run(P, opts, rho_d, f_d, u_d, reps=3):
    """The 2D step with the paper's outer solver, flexible GMRES(30), instead of flexible CG
    (host-driven: the Givens rotations run on the host)."""
    import torch
    o = dict(opts, krylov="fgmres", gmres_restart=30)
    times, its = [], []
    for k in range(reps + 1):
        u_d.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.set_density(rho_d)
        P.setup(prec="fp32", **o)
        _, res = P.solve(f_d, u0=u_d)
        torch.cuda.synchronize()
        if k:
            times.append(time.perf_counter() - t0)
            its.append(res[0]["iterations"])
    return {"solves_per_s": 1.0 / statistics.median(times), "iterations": statistics.median(its),
            "rel_residual": res[0]["rel_residual"], "restart": 30,
            "timing": "host clock around set_density + setup + solve (the solve synchronises)"}


def design_run(P, opts, p, rho_d, f_d, iters=5):
    """Design iterations around the solve (Sec. 2.1), all on the device: rho = S alpha, SIMP
    moduli, hierarchy setup, the solve warm-started from the previous design's u, the
    sensitivities dF/drho and dF/dalpha = S^T dF/drho.  alpha is perturbed by seeded 5 % noise
    between iterations (no optimiser: MMA is out of scope)."""
    import torch
    g = torch.Generator(device=rho_d.device)
    g.manual_seed(7)
    alpha = rho_d.clone()
    u = torch.zeros_like(f_d)
    times, its, rel = [], [], []
    for k in range(iters + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rho = P.density_filter(alpha)
        P.set_density(rho)
        P.setup(prec="fp32", **opts)
        u, res = P.solve(f_d, u0=u)
        dc = P.compliance_sensitivity(u)
        da = P.density_filter(dc, transpose=True)
        torch.cuda.synchronize()
        if k:
            times.append(time.perf_counter() - t0)
            its.append(res[0]["iterations"])
            rel.append(res[0]["rel_residual"])
        alpha = torch.clamp(alpha * (1 + 0.05 * (2 * torch.rand(alpha.shape, generator=g,
                                                                device=alpha.device,
                                                                dtype=alpha.dtype) - 1)), 1e-3, 1.0)
    return {"ms_per_iteration": 1e3 * statistics.median(times), "iterations": its,
            "rel_residual": rel,
            "converged_to_1e-8": int(sum(r <= 1e-8 for r in rel)),
            "note": "filtered densities grade the 1e9 contrast; the FP64 oracle PCG also stalls "
                    "near 2e-8 on the filtered design (757 iterations): solves that stop above "
                    "1e-8 are reported as such, not counted as converged",
            "steps": "filter, moduli, setup, warm-started solve, sensitivities, filter transpose",
            "sensitivity_sum": float(da.sum().item())}


def stability_run(tomg, ctx, opts, nx=256, ny=1024):
    """The stability problem on the paper's 2D column (256 x 1024 quad4, about 526k DOFs;
    seeded smoothed density in [0.1, 1]), every step on the device: setup, the displacement
    solve, the six largest buckling eigenpairs by generalized Davidson (j_min 10, j_max 25,
    tol 1e-6, the V-cycle as preconditioner), the six adjoint right-hand sides
    Phi^T (dK_sigma/du) Phi, the six adjoint solves on concurrent slots from zero, and the
    sensitivities of the p = 8 norm of the eigenvalues with the filter transpose."""
    import torch
    import workloads as W
    p = W.column_2d(nx, ny, seed=0)
    P = tomg.Problem.from_workload(ctx, p)
    o = dict(opts, concurrency=6)
    f = torch.from_numpy(p.f).cuda()
    phases = {"setup": [], "solve": [], "davidson": [], "adjoint_rhs": [], "adjoint_solves": [],
              "sensitivities": []}
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.setup(prec="fp32", **o)
        t1 = time.perf_counter()
        u, res = P.solve(f)
        t2 = time.perf_counter()
        lam, Phi, it, st = P.buckling(u[0], n_eig=6, tol=1e-6, modes=True)
        t3 = time.perf_counter()
        g = P.buckling_adjoint_rhs(Phi)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        v, ra = P.solve(g)
        t5 = time.perf_counter()
        _, dF, F = P.buckling_sensitivity(u[0], lam, Phi, v, pnorm=8, per_mode=False)
        da = P.density_filter(dF, radius=1.5, transpose=True)
        torch.cuda.synchronize()
        t6 = time.perf_counter()
        if k:
            for name, a, b in (("setup", t0, t1), ("solve", t1, t2), ("davidson", t2, t3),
                               ("adjoint_rhs", t3, t4), ("adjoint_solves", t4, t5),
                               ("sensitivities", t5, t6)):
                phases[name].append(1e3 * (b - a))
    return {"workload": "2D column quad4 %dx%d (%d DOFs), bottom clamped, unit load on top" %
                        (nx, ny, p.n),
            "ms": {k: statistics.median(v) for k, v in phases.items()},
            "lambdas": [float(x) for x in lam], "pnorm8": F,
            "davidson_iterations": it, "davidson_status": st,
            "solve_iterations": res[0]["iterations"],
            "adjoint_iterations": [r["iterations"] for r in ra],
            "adjoint_rel_residual_max": max(r["rel_residual"] for r in ra),
            "dF_dalpha_sum": float(da.sum().item()),
            "timing": "host clock per phase, device arrays throughout, synchronised per phase"}


def batched_run(tomg, ctx, slots, reps=3, prec="tc", smoother="chebyshev", cheb_degree=2):
    """The 16 right-hand sides (8 point loads, 8 adjoint-like vectors) of the 3D hex8 128x64x64
    case (1,635,075 DOFs) on one shared hierarchy: as one block solve (every kernel launch
    covers all 16), on `slots` concurrent solve slots, and one after another (one slot).
    Median of `reps` runs, setup excluded; the right-hand sides and solutions stay in device
    memory (as for the headline's `value`), so that page faults of fresh host arrays do not enter
    the times; every right-hand side compared with the oracle's reference."""
    import torch
    import refs
    import workloads as W
    p = W.batched_3d()
    P = tomg.Problem.from_workload(ctx, p)
    ref = refs.load("batched3d_128x64x64")
    G = refs.projections(p.n)
    f_dev = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
    u_dev = torch.zeros_like(f_dev)
    res = {}
    for conc in ("block", slots, 1):
        block = p.nrhs if conc == "block" else 0
        P.setup(pc="hybrid", prec=prec, n_geo_levels=3, max_coarse_dofs=1000, rtol=1e-8,
                concurrency=1 if conc == "block" else conc, block_rhs=block, smoother=smoother,
                cheb_degree=cheb_degree)
        u_dev.zero_()
        torch.cuda.synchronize()
        P.solve(f_dev, out=u_dev)  # warm-up: graphs and vectors of the slots or the block
        times, worst_rr = [], 0.0
        for _ in range(reps):
            u_dev.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, r = P.solve(f_dev, out=u_dev)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            its = [x["iterations"] for x in r]
            worst_rr = max(worst_rr, max(x["rel_residual"] for x in r))
        u = u_dev.cpu().numpy()
        t = statistics.median(times)
        res[conc] = {"solves_per_s": p.nrhs / t, "ms_all_rhs": 1e3 * t,
                     "iterations_median": statistics.median(its), "rel_residual_max": worst_rr,
                     "setup_ms": r[0]["setup_ms"],
                     "accuracy_worst_rhs": worst([accuracy_of(u[j], r[j], ref[j], G)
                                                  for j in range(p.nrhs)])}
    # the level-0 FP32 kernels of this case timed alone (cold L2, CUDA events), with the
    # minimum-traffic bytes of one launch
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    kern = {}
    for name in ("residual", "jacobi"):
        for kp in ("tc", "fp32"):
            ms = P.time_fine_operator(name, kp, reps=20, cold_l2=True)
            nb = kernel_bytes(name, kp, p)
            kern["%s_%s" % (name, kp)] = {
                "kernel": "k_ebe3tc (tcgen05 kind::f16, split x against integer Ke)" if kp == "tc" else "k_ebe3 (CUDA cores)",
                "ms_per_launch": ms, "algorithmic_bytes": nb,
                "achieved_gbs": nb / (ms * 1e-3) / 1e9, "frac_hbm": nb / (ms * 1e-3) / 1e9 / hbm,
                "element_gflops": 1152.0 * p.nel / (ms * 1e-3) / 1e9}
    P.close()
    return {"workload": "3D cantilever hex8 128x64x64 (1,635,075 DOFs), 8 point loads + 8 "
                        "adjoint-like right-hand sides, hybrid hierarchy, FP32 V-cycle with "
                        "tensor-core element contractions",
            "rhs": p.nrhs,
            "block": dict(res["block"], mode="one block solve: every launch covers all %d "
                                              "right-hand sides" % p.nrhs),
            "concurrent": dict(res[slots], slots=slots), "one_at_a_time": res[1],
            "level0_kernels": kern}


def serving_run(tomg, ctx, n_clients, n_updates, slots, budget_gb=160):
    """The serving stream: `n_clients` topology-optimisation clients arrive as a Poisson stream
    (50 per second), each on a grid drawn uniformly from 2D 64x32 .. 1024x512 and 3D 32x16x16 ..
    192x96x96 (doubling steps).  A client submits its next design (5 % seeded noise on the
    previous one) as soon as the previous solve returns (warm-started on the device from the
    previous displacements), `n_updates` designs in all, then retires its problem.  The server
    admits requests by device-memory budget (problems between their updates stay resident and
    count against it) and overlaps up to `slots` of them on the GPU."""
    import workloads as W
    stream = W.serving_stream(n_requests=n_clients, n_updates=n_updates)
    opt = dict(pc="hybrid", prec="tc", n_geo_levels=3, max_coarse_dofs=1000, concurrency=1,
               max_iter=2000)
    srv = tomg.Server(ctx, budget_gb << 30, slots)
    lock = threading.Lock()
    stats = {"solves": 0, "converged": 0, "not_converged_rel_residual": [], "errors": []}

    def client(r):
        try:
            p = W.serving_problem(r, 0)
            P = tomg.Problem(ctx, p.dim, p.nx, p.ny, p.nz, p.E0, p.Emin, p.penal, p.nu)
            P.set_fixed_dofs(p.fixed)
            rho = W.serving_density(r, 0)
            rng = np.random.default_rng(r["field_seed"] + 100000)
            for k in range(n_updates):
                if k:
                    rho = np.clip(rho * (1.0 + r["noise"] * rng.standard_normal(rho.shape)),
                                  1e-3, 1.0)
                res = srv.wait(srv.submit(P, rho, p.f[0], **opt), timeout_ms=300000)[0]
                with lock:
                    stats["solves"] += 1
                    if res["status"] == 0 and res["rel_residual"] <= 1e-8:
                        stats["converged"] += 1
                    else:
                        stats["not_converged_rel_residual"].append(res["rel_residual"])
            srv.retire(P, timeout_ms=300000)
            P.close()
        except Exception as e:  # noqa: BLE001
            with lock:
                stats["errors"].append(str(e)[:200])

    threads = []
    t0 = time.perf_counter()
    for r in stream:
        wait = r["t_arrive"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        th = threading.Thread(target=client, args=(r,), daemon=True)
        th.start()
        threads.append(th)
    for th in threads:
        th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    dofs = sorted({W.n_dofs(r["dim"], r["nx"], r["ny"], r["nz"]) for r in stream})
    return {"clients": n_clients, "updates_per_client": n_updates, "slots": slots,
            "solves": stats["solves"], "solves_per_s": stats["solves"] / wall,
            "wall_s": wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "peak_active": st["peak_active"], "peak_device_gb": st["peak_bytes"] / 2 ** 30,
            "budget_gb": budget_gb,
            "converged_to_1e-8": stats["converged"],
            "not_converged_rel_residual": sorted(stats["not_converged_rel_residual"])[-8:],
            "errors": stats["errors"][:4], "dofs_min": dofs[0], "dofs_max": dofs[-1],
            "preconditioner": "hybrid (3 geometric levels + SA-AMG < 1000 DOFs), FP32 V-cycle",
            "arrivals": "Poisson, 50 clients/s; each client's next design is submitted when its "
                        "previous solve returns (closed loop), warm-started on the device"}


FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 rate (nominal; the measured-peaks file has no FP64 figure)
# the method's work per DOF of one operator application (hex8: 1152 flops per element)
MODEL_FLOPS_PER_DOF = {2: 64.0, 3: 384.0}


def roofline(P, p, head, opts):
    """The level-0 kernels of one FCG iteration of the headline, each timed live on the context
    stream with CUDA events (cold L2 before each launch): the FP64 outer q = K p (+ dot) on the
    tensor cores (exact digit products, k_ebe3x64), and the V-cycle's FP32 residual and
    Chebyshev / Jacobi steps on the FP32 tensor-core element operator (k_ebe3tc).  The dominant
    kernel is the one with the largest share of the solve (time per launch x launches per
    iteration).  The FP64 outer apply it replaces, on the assembled 3^d stencil, is timed beside
    it (a setup with fp64_tc = 0)."""
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    src = "measured" if "fallback" not in peaks else "fallback"
    nn = p.n // p.dim
    out = {}
    # launches per outer iteration: one outer apply; degree-2 Chebyshev V-cycle on level 0:
    # one smoothing step before and two after the coarse correction, one residual
    per_it = {"outer": 1, "residual": 1, "jacobi": 3}
    for name, prec in (("outer", "fp64"), ("residual", HEAD_PREC), ("jacobi", HEAD_PREC)):
        ms = P.time_fine_operator(name, prec, reps=20, cold_l2=True)
        b = kernel_bytes(name, prec, p)
        out[name] = {"ms_per_launch": ms, "algorithmic_bytes": b, "launches_per_iteration":
                     per_it[name], "achieved_gbs": b / (ms * 1e-3) / 1e9,
                     "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm}
    o = out["outer"]
    o["kernel"] = "k_ebe3x64 (FP64 outer q = K p + p.q; exact 11-bit digit products on the " \
                  "FP16 tensor cores)"
    model = MODEL_FLOPS_PER_DOF[p.dim] * p.n
    o["model_flops"] = model
    o["fp64_equivalent_tflops"] = model / (o["ms_per_launch"] * 1e-3) / 1e12
    # MMA work as issued: per element row 5 digits x (K 32 x N 32) multiply-adds; the tiles
    # partition the elements, one row per element
    rows = p.nel
    o["tensor_tflops_issued"] = rows * 5 * 32 * 32 * 2 / (o["ms_per_launch"] * 1e-3) / 1e12
    o["tensor_frac_of_bf16_peak"] = o["tensor_tflops_issued"] / bf16
    # the assembled FP64 stencil it replaces
    P.setup(prec=HEAD_PREC, **dict(opts, fp64_tc=0))
    ms_st = P.time_fine_operator("outer", "fp64", reps=20, cold_l2=True)
    executed = 2 * nn * (3 ** p.dim) * p.dim * p.dim + 2 * p.n
    out["outer_fp64_stencil"] = {
        "kernel": "k_stencil_apply_dot<%d> (assembled 3^d FP64 stencil)" % p.dim,
        "ms_per_launch": ms_st, "executed_flops": executed,
        "executed_tflops": executed / (ms_st * 1e-3) / 1e12,
        "frac_fp64_peak": executed / (ms_st * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
        "stencil_bytes": nn * (3 ** p.dim) * p.dim * p.dim * 8 + 2 * 8 * p.n + nn,
        "stencil_frac_hbm": (nn * (3 ** p.dim) * p.dim * p.dim * 8 + 2 * 8 * p.n + nn)
                            / (ms_st * 1e-3) / 1e9 / hbm,
        "launches_per_iteration": 0}
    P.setup(prec=HEAD_PREC, **opts)
    dom = max((k for k in out if out[k]["launches_per_iteration"]),
              key=lambda k: out[k]["ms_per_launch"] * out[k]["launches_per_iteration"])
    k = out[dom]
    bytes_counted = ("minimum traffic of the work model: x and y (and b, the block inverse) "
                     "once, one modulus per element, one mask byte per node")
    headr = {"kernel": k.get("kernel", "k_ebe3tc (%s, FP32 on the tensor cores)" % dom),
             "bound": "hbm", "achieved": k["achieved_gbs"], "peak": hbm, "unit": "GB/s",
             "frac": k["frac_hbm"], "peak_source": src, "bytes_counted": bytes_counted}
    if dom == "outer":
        # the work model's two lower bounds on one FP64 apply: its bytes at the HBM rate and its
        # flops (384 per DOF for hex8, 64 for quad4) at the FP64 rate; the larger one binds
        t_hbm = k["algorithmic_bytes"] / (hbm * 1e9)
        t_fp64 = o["model_flops"] / (FP64_PEAK_TFLOPS * 1e12)
        if t_fp64 > t_hbm:
            headr.update({"bound": "alu", "achieved": o["fp64_equivalent_tflops"],
                          "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": o["fp64_equivalent_tflops"] / FP64_PEAK_TFLOPS,
                          "peak_source": "nominal GB300 FP64 rate (no measured FP64 figure)",
                          "flops_counted": "the method's FP64 work, %d flops per DOF"
                                           % MODEL_FLOPS_PER_DOF[p.dim],
                          "bound_times_ms": {"fp64_flops": t_fp64 * 1e3, "hbm_bytes": t_hbm * 1e3},
                          "hbm": {"achieved": k["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                                  "frac": k["frac_hbm"], "peak_source": src,
                                  "bytes_counted": bytes_counted}})
            del headr["bytes_counted"]
        headr["note"] = ("the FP64 products run exactly on the FP16 tensor cores (11-bit digits), "
                         "so the kernel is not held to the FP64 pipe's rate: FP64-equivalent %.2f "
                         "TFLOP/s, %.2f x GB300's FP64 rate; its own binding unit is the FP64 pipe "
                         "that converts and scales the integer products; the assembled FP64 "
                         "stencil it replaces runs at %.2f of the FP64 rate and takes %.3f ms"
                         % (o["fp64_equivalent_tflops"],
                            o["fp64_equivalent_tflops"] / FP64_PEAK_TFLOPS,
                            out["outer_fp64_stencil"]["frac_fp64_peak"], ms_st))
    share = {kk: out[kk]["ms_per_launch"] * out[kk]["launches_per_iteration"] * head["iterations"]
             / head["solve_ms"] for kk in out if out[kk]["launches_per_iteration"]}
    headr.update({"traffic": TRAFFIC.get((dom, p.dim, p.n)),
                  "ms_per_launch": k["ms_per_launch"], "share_of_solve": share, "kernels": out})
    return headr


# DRAM read + write bytes of one launch, from the ncu captures summarised under profiles/
# (key: kernel role, dimension, DOFs); valid while the kernel is unchanged since its capture
TRAFFIC = {
    # the FP64 tensor-core apply, 3D cantilever 192x96x96: tile kernel 59.6 MB read + 9.7 MB
    # write, node kernel 107.1 MB read + 16.0 MB write (means of two applies)
    ("outer", 3, 5447811): 192.4e6,
}


def kernel_only(args):
    """One level-0 operator kernel timed alone (cold L2 before each launch, CUDA events on the
    context stream), with its algorithmic bytes per launch."""
    import torch
    import workloads as W
    from paper_2001_01655_gb300 import tomg

    dims = [int(v) for v in args.kernel_grid.lower().split("x")]
    p = W.cantilever_2d(nx=dims[0], ny=dims[1], seed=0) if len(dims) == 2 else \
        W.cantilever_3d(nx=dims[0], ny=dims[1], nz=dims[2], seed=0)
    ctx = tomg.Context(0)
    P = tomg.Problem.from_workload(ctx, p)
    prec = "fp64" if args.kernel == "outer" else args.kernel_prec
    P.setup(pc="gmg", prec=prec, max_coarse_dofs=8000)
    ms = P.time_fine_operator(args.kernel, prec, reps=args.kernel_reps, cold_l2=True)
    nbytes = kernel_bytes(args.kernel, prec, p)
    peaks = load_peaks()
    torch.cuda.synchronize()
    return {"kernel": args.kernel, "prec": prec, "grid": dims, "dofs": p.n, "ms_per_launch": ms,
            "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
            "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6800.0)}


def kernel_bytes(kernel, prec, p):
    """Algorithmic bytes of one level-0 operator launch: the vectors it must read and write,
    one modulus per element and one mask byte per node (the minimum-traffic model)."""
    s = 8 if prec == "fp64" else 4
    nn = p.n // p.dim
    vec = {"outer": 2, "apply": 2, "residual": 3, "jacobi": 3}[kernel]
    extra = p.dim * s * nn if kernel == "jacobi" else 0  # block-diagonal inverse, dim^2 per node
    return vec * s * p.n + s * p.nel + nn + extra


def _cpu_seconds():
    import resource
    r = resource.getrusage(resource.RUSAGE_SELF)
    return r.ru_utime + r.ru_stime


def oracle_solve_timed(p, smoother="chebyshev"):
    """One complete oracle solve of problem p as the bench times it on the GPU: SIMP moduli,
    assembly, the hybrid hierarchy (3 geometric levels, SA-AMG to < 1000 DOFs), FP64 PCG from
    u = 0 to a true relative residual of 1e-8.  Returns (seconds, iterations, rel. residual)."""
    from oracle import solve as osolve
    t0 = time.perf_counter()
    r = osolve.solve(p, pc="hybrid", n_geo=3, cap=1000, rtol=1e-8, max_iter=2000,
                     smoother=smoother)
    return time.perf_counter() - t0, int(r["iterations"][0]), float(r["rel_residual"][0])


def cpu_baseline(steps=3, warmup=0, smoother="chebyshev"):
    """The oracle (plain FP64 numpy / scipy) on the host cores: complete solves (setup and PCG
    to 1e-8) of the same cantilever recipe at SAMPLE_GRID (1/27 of the elements), timed in
    this run; solves/s of the headline workload = that rate / the DOF ratio (the oracle's setup
    and its iterations are linear in the DOF count, and its iteration count barely changes
    with the grid: 20 to 1e-12 at 192x96x96, 19 at 48x24x24).  `cores` is the CPU time over
    the wall time (the threads BLAS and scipy kept busy)."""
    import workloads as W
    ps = W.cantilever_3d(*SAMPLE_GRID, seed=WORKLOAD["seed"])
    n_full = W.n_dofs(3, WORKLOAD["nx"], WORKLOAD["ny"], WORKLOAD["nz"])
    ratio = n_full / ps.n
    for _ in range(warmup):
        oracle_solve_timed(ps, smoother)
    c0, t0 = _cpu_seconds(), time.perf_counter()
    secs, its, rr = [], [], []
    for _ in range(steps):
        s, i, r = oracle_solve_timed(ps, smoother)
        secs.append(s)
        its.append(i)
        rr.append(r)
    wall = time.perf_counter() - t0
    cores = (_cpu_seconds() - c0) / wall
    s = statistics.median(secs)
    return {"value": 1.0 / (s * ratio), "unit": "solves/s", "cores": round(cores, 1),
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d complete oracle solves (setup + FP64 PCG to 1e-8, %d iterations, "
                      "true residual %.1e; %s smoother) of the same cantilever at %dx%dx%d "
                      "(%d DOFs): %.2f s each (median), scaled by the DOF ratio %.1f"
                      % (steps, statistics.median(its), max(rr), smoother, *SAMPLE_GRID, ps.n,
                         s, ratio),
            "sample_solves_per_s": 1.0 / s, "sample_dofs": ps.n, "sample_grid": list(SAMPLE_GRID),
            "step_seconds": secs, "iterations": statistics.median(its)}


def gpu_on_sample(args):
    """The headline configuration on the oracle's sample grid, for a same-size comparison."""
    import torch
    import workloads as W
    from paper_2001_01655_gb300 import tomg
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = tomg.Context(0, stream)
    p = W.cantilever_3d(*SAMPLE_GRID, seed=WORKLOAD["seed"])
    S = Stepper(tomg, ctx, p, stream, dev)
    opts = dict(HEADLINE, use_graph=args.graph_mode, smoother=args.smoother,
                cheb_degree=args.cheb_degree)
    t, r, _ = S.timed(HEAD_PREC, opts, 10, 3)
    return S.summary(t, r)["solves_per_s"]


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only; each step is one complete oracle solve of
    the sample grid (W untimed first), and the value is scaled to the headline workload as in
    cpu_baseline.  ms_per_step is the measured time of one such step."""
    if rank != 0:
        return None
    cb = cpu_baseline(steps=args.steps, warmup=args.warmup, smoother=args.smoother)
    value = cb["value"]
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(cb["step_seconds"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_label(),
                       "preconditioner": "hybrid: 3 geometric levels, SA-AMG below to < 1000 DOFs",
                       "rtol": 1e-8, "smoother": smoother_label(args)},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "host_cores", "kind",
                                                "sample")},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.kernel:
        print(json.dumps(kernel_only(args)))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)  # host only; ranks other than 0 do nothing
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_gpu(args, rank, world, local)
    if rank == 0 and world == 1 and not args.no_cpu:
        progress("cpu baseline")
        cb = cpu_baseline(smoother=args.smoother)
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "host_cores", "kind",
                                                  "sample", "sample_solves_per_s")}
        out["cpu_baseline"]["gpu_solves_per_s_on_sample"] = gpu_on_sample(args)
    if rank == 0 and out is not None:
        progress("done")
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
