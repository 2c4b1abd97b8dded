"""Throughput of the multigrid-preconditioned CG solve of the SIMP elasticity system.

One step = one whole pass of the hot path on the 2D cantilever (768 x 384 quad4 elements,
592,130 DOFs, thin 0/1 members with 1e9 stiffness contrast): SIMP moduli from the density
already resident in HBM, preconditioner setup (Galerkin hierarchy, smoother blocks, coarse
Cholesky), and a solve to a true relative residual of 1e-8.  Headline: mixed precision
(FP32 V-cycle inside FP64 flexible CG); the FP64 V-cycle PCG is measured beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  The reference arm times the CPU oracle (plain FP64 numpy /
scipy PCG with the same kind of hierarchy) on a bounded sample of the same workload.
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

METRIC = "MG-PCG solves/sec & DOF-iters/sec @1e-8 residual, mixed vs FP64; p50/p99 latency"
WORKLOAD = dict(nx=768, ny=384, seed=0)
HEADLINE = dict(pc="hybrid", max_coarse_dofs=1500, n_geo_levels=2)


def smoother_label(args):
    if args.smoother == "chebyshev":
        return "chebyshev degree %d" % args.cheb_degree
    if args.smoother == "gmres":
        return "gmres 2 steps per smoothing"
    return args.smoother


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tomg")
    ap.add_argument("--pc", default=HEADLINE["pc"])
    ap.add_argument("--cap", type=int, default=HEADLINE["max_coarse_dofs"])
    ap.add_argument("--n-geo", type=int, default=HEADLINE["n_geo_levels"])
    ap.add_argument("--graph-mode", type=int, default=2,
                    help="2: whole solve in one graph (device while loop); 1: one graph per "
                         "iteration (host polls); 0: no graphs")
    ap.add_argument("--serving", type=int, default=24,
                    help="requests of the mixed-size serving stream replayed after the main "
                         "measurement (0: skip)")
    ap.add_argument("--serving-updates", type=int, default=2)
    ap.add_argument("--batched", type=int, default=1,
                    help="also time the 16 right-hand sides of the 3D 128x64x64 case (0: skip)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--smoother", default="chebyshev", choices=["jacobi", "chebyshev", "gmres"],
                    help="V-cycle smoother of the timed solves; the paper's runs use one Jacobi "
                         "sweep, which is measured beside the headline as `jacobi` (and the "
                         "GMRES smoother as `gmres_smoother`)")
    ap.add_argument("--cheb-degree", type=int, default=2)
    ap.add_argument("--batched-prec", default="tf32x3", choices=["fp32", "tf32x3"],
                    help="V-cycle precision of the batched 3D measurement: fp32 CUDA-core or "
                         "3xTF32 tensor-core element contractions")
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


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


def run_gpu(args, rank, world, local):
    import torch
    import workloads as W
    from paper_2001_01655_gb300 import tomg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    ctx = tomg.Context(local, stream)
    p = W.cantilever_2d(**WORKLOAD)
    P = tomg.Problem.from_workload(ctx, p)
    rho_d = torch.tensor(p.rho, dtype=torch.float64, device=dev)
    f_d = torch.tensor(p.f[0], dtype=torch.float64, device=dev)
    u_d = torch.zeros_like(f_d)
    flush = torch.empty(256 << 20, dtype=torch.int8, device=dev)  # 256 MB > 129 MB L2
    opts = dict(pc=args.pc, max_coarse_dofs=args.cap, n_geo_levels=args.n_geo, rtol=1e-8,
                max_iter=2000, use_graph=args.graph_mode, smoother=args.smoother,
                cheb_degree=args.cheb_degree)

    def step(prec, o=None):
        u_d.zero_()
        P.set_density(rho_d)
        P.setup(prec=prec, **(o or opts))
        _, res = P.solve(f_d, u0=u_d)
        return res[0]

    def timed(prec, K, Wm, o=None):
        for _ in range(Wm):
            step(prec, o)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times, its, results = [], [], []
        l0 = ctx.kernel_launches()
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = step(prec, o)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            its.append(r["iterations"])
            results.append(r)
        launches = ctx.kernel_launches() - l0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return times, its, results, launches

    with Clocks(local) as clk:
        times, its, results, launches = timed("fp32", args.steps, args.warmup)
    total_ms = max_over_ranks(sum(times), world, device=dev)
    bad = [r for r in results if r["status"] != 0 or r["rel_residual"] > 1e-8]
    out = {
        "metric": METRIC,
        "value": throughput(args.steps, world, total_ms),
        "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 outer / f32 V-cycle", "data": "synthetic",
        "config": {"workload": "2D cantilever quad4 %dx%d (592,130 DOFs), seeded thin 0/1 members "
                   "(1e9 contrast), left edge clamped, unit load right mid-edge" % (WORKLOAD["nx"], WORKLOAD["ny"]),
                   "preconditioner": args.pc, "max_coarse_dofs": args.cap, "rtol": 1e-8,
                   "smoother": smoother_label(args),
                   "step": "SIMP moduli + hierarchy setup + FCG solve from u = 0",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "dof_iters_per_s": world * p.n * sum(its) / (total_ms / 1e3),
        "iterations": statistics.median(its),
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
        "setup_ms": statistics.median(r["setup_ms"] for r in results),
        "solve_ms": statistics.median(r["solve_ms"] for r in results),
        "rel_residual_max": max(r["rel_residual"] for r in results),
        "failed_steps": len(bad),
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_fp64:
        t64, i64, r64, _ = timed("fp64", max(3, args.steps // 2), 1)
        out["fp64"] = {"solves_per_s": len(t64) / (sum(t64) / 1e3),
                       "dof_iters_per_s": p.n * sum(i64) / (sum(t64) / 1e3),
                       "iterations": statistics.median(i64),
                       "setup_ms": statistics.median(r["setup_ms"] for r in r64),
                       "solve_ms": statistics.median(r["solve_ms"] for r in r64)}
    if args.smoother != "jacobi" and not args.no_fp64:
        # the paper's smoother (one weighted point-block Jacobi sweep), mixed and FP64
        oj = dict(opts, smoother="jacobi")
        jac = {}
        for prec in ("fp32", "fp64"):
            tj, ij, rj, _ = timed(prec, max(3, args.steps // 2), 1, oj)
            jac["mixed" if prec == "fp32" else "fp64"] = {
                "solves_per_s": len(tj) / (sum(tj) / 1e3), "iterations": statistics.median(ij),
                "setup_ms": statistics.median(r["setup_ms"] for r in rj),
                "solve_ms": statistics.median(r["solve_ms"] for r in rj),
                "rel_residual_max": max(r["rel_residual"] for r in rj)}
        out["jacobi"] = jac
        # the paper's third smoother (Sec. 4.1): GMRES steps per smoothing, flexible CG outside
        gm = {}
        for steps_ in (2, 4):
            og = dict(opts, smoother="gmres", gmres_steps=steps_)
            tg, ig, rg, _ = timed("fp32", max(3, args.steps // 2), 1, og)
            gm["steps_%d" % steps_] = {
                "solves_per_s": len(tg) / (sum(tg) / 1e3), "iterations": statistics.median(ig),
                "solve_ms": statistics.median(r["solve_ms"] for r in rg),
                "rel_residual_max": max(r["rel_residual"] for r in rg)}
        out["gmres_smoother"] = gm
    # end to end through the C ABI with host buffers (copies inside the timed region)
    rho_h, f_h = p.rho.copy(), p.f[0].copy()
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.set_density(rho_h)
        P.setup(prec="fp32", **opts)
        u_h, res = P.solve(f_h, u0=np.zeros_like(f_h))
        e2e.append(time.perf_counter() - t0)
    out["e2e"] = {"value": world / statistics.median(e2e), "unit": "solves/s",
                  "h2d_bytes_per_step": int(rho_h.nbytes + 2 * f_h.nbytes),
                  "d2h_bytes_per_step": int(f_h.nbytes)}
    out["roofline"] = roofline(P, ctx, p, stream)
    if not args.no_fp64:
        out["fgmres"] = fgmres_run(P, opts, rho_d, f_d, u_d, stream)
        out["design_iteration"] = design_run(P, opts, p, rho_d, f_d, stream)
        out["stability"] = stability_run(tomg, ctx, opts)
    if args.serving > 0:
        out["serving"] = serving_run(tomg, ctx, args.serving, args.serving_updates, args.slots)
    if args.batched:
        out["batched"] = batched_run(tomg, ctx, args.slots, prec=args.batched_prec,
                                     smoother=args.smoother, cheb_degree=args.cheb_degree)
    return out


def fgmres_run(P, opts, rho_d, f_d, u_d, stream, reps=3):
    """The headline step with the paper's outer solver, flexible GMRES(30), instead of flexible
    CG (host-driven: the Givens rotations run on the host)."""
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


def design_run(P, opts, p, rho_d, f_d, stream, iters=5):
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
            "note": "filtered densities grade the 1e9 contrast; the FP64 oracle PCG also stalls "
                    "near 2e-8 on the filtered design (757 iterations), so these solves stop at "
                    "max_iter slightly above 1e-8",
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


def batched_run(tomg, ctx, slots, reps=3, prec="tf32x3", smoother="jacobi", cheb_degree=2):
    """The 16 right-hand sides (8 point loads, 8 adjoint-like vectors) of the 3D hex8 128x64x64
    case (1,635,075 DOFs) on one shared hierarchy: all 16 on `slots` concurrent solve slots,
    against the same 16 one after another (one slot).  Median of `reps` runs, setup excluded."""
    import workloads as W
    p = W.batched_3d()
    P = tomg.Problem.from_workload(ctx, p)
    res = {}
    for conc in (slots, 1):
        P.setup(pc="hybrid", prec=prec, n_geo_levels=3, max_coarse_dofs=1000, rtol=1e-8,
                concurrency=conc, smoother=smoother, cheb_degree=cheb_degree)
        P.solve(p.f[:2])  # warm-up: graphs and vectors of the slots
        times, its, worst = [], [], 0.0
        for _ in range(reps):
            t0 = time.perf_counter()
            _, r = P.solve(p.f)
            times.append(time.perf_counter() - t0)
            its = [x["iterations"] for x in r]
            worst = max(worst, max(x["rel_residual"] for x in r))
        t = statistics.median(times)
        res[conc] = {"solves_per_s": p.nrhs / t, "ms_all_rhs": 1e3 * t,
                     "iterations_median": statistics.median(its), "rel_residual_max": worst,
                     "setup_ms": r[0]["setup_ms"]}
    # the level-0 FP32 kernels of this case timed alone (cold L2, CUDA events), with the
    # minimum-traffic bytes of one launch
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    kern = {}
    for name in ("residual", "jacobi"):
        for kp in ("tf32x3", "fp32"):
            ms = P.time_fine_operator(name, kp, reps=20, cold_l2=True)
            nb = kernel_bytes(name, kp, p)
            kern["%s_%s" % (name, kp)] = {
                "kernel": "k_ebe3tc (tcgen05 3xTF32)" if kp == "tf32x3" else "k_ebe3 (CUDA cores)",
                "ms_per_launch": ms, "algorithmic_bytes": nb,
                "achieved_gbs": nb / (ms * 1e-3) / 1e9, "frac_hbm": nb / (ms * 1e-3) / 1e9 / hbm,
                "element_gflops": 1152.0 * p.nel / (ms * 1e-3) / 1e9}
    res["kernels"] = kern
    return {"workload": "3D cantilever hex8 128x64x64 (1,635,075 DOFs), 8 point loads + 8 "
                        "adjoint-like right-hand sides, hybrid hierarchy, %s V-cycle" %
                        ("FP32 (3xTF32 tensor-core element contractions)" if prec == "tf32x3"
                         else "FP32"),
            "rhs": p.nrhs, "concurrent": dict(res[slots], slots=slots), "one_at_a_time": res[1],
            "level0_kernels": res["kernels"]}


def serving_run(tomg, ctx, n_requests, n_updates, slots):
    """Replay the mixed 2D/3D request stream (Poisson arrivals, 5 % density noise per update)
    through the continuous-batching server; every update of a request is submitted at the
    request's arrival time and warm-starts from the previous one on the device."""
    import workloads as W
    stream = W.serving_stream(n_requests=n_requests, n_updates=n_updates)
    opt = dict(pc="hybrid", prec="tf32x3", n_geo_levels=3, max_coarse_dofs=1000, concurrency=1,
               max_iter=2000)
    probs = []
    for r in stream:
        p = W.serving_problem(r, 0)
        P = tomg.Problem(ctx, p.dim, p.nx, p.ny, p.nz, p.E0, p.Emin, p.penal, p.nu)
        P.set_fixed_dofs(p.fixed)
        dens = [W.serving_density(r, k) for k in range(n_updates)]
        probs.append((P, p, dens))
    srv = tomg.Server(ctx, 64 << 30, slots)
    t0 = time.perf_counter()
    tickets = []
    for (P, p, dens), r in zip(probs, stream):
        wait = r["t_arrive"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        for k in range(n_updates):
            tickets.append(srv.submit(P, dens[k], p.f[0], **opt))
    statuses = [srv.wait(t)[0]["status"] for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    dofs = sorted({p.n for _, p, _ in probs})
    return {"requests": n_requests, "updates_per_request": n_updates, "slots": slots,
            "solves": len(tickets), "solves_per_s": len(tickets) / wall,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "peak_active": st["peak_active"],
            "converged": int(sum(s == 0 for s in statuses)), "dofs_min": dofs[0],
            "dofs_max": dofs[-1], "preconditioner": "hybrid (3 geometric levels + SA-AMG < 1000 DOFs)",
            "arrivals": "Poisson, 50 requests/s; each request's updates queued on arrival"}


FP64_PEAK_GFLOPS = 1250.0  # GB300 FP64 rate (nominal, not in the measured peaks file)
# DRAM read + write of one k_stencil_apply_dot<2> launch on this workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, caches flushed before the launch)
OUTER_TRAFFIC_BYTES = 89912320 + 2731264


def roofline(P, ctx, p, stream):
    """The level-0 kernels of one FCG iteration, each timed live on the context stream with CUDA
    events (cold L2 before each launch): the FP64 outer q = K p (+ dot) on the assembled fine
    stencil, and the V-cycle's FP32 residual and Jacobi sweeps on the element operator.  The
    slowest is the dominant kernel; its roofline is the bound that binds it."""
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "measured" if "fallback" not in peaks else "fallback"
    nn = p.n // p.dim
    out = {}
    for name, prec in (("outer", "fp64"), ("residual", "fp32"), ("jacobi", "fp32")):
        try:
            ms = P.time_fine_operator(name, prec, reps=50, cold_l2=True)
        except Exception as e:  # noqa: BLE001
            return {"error": str(e)}
        b = kernel_bytes(name, prec, p)
        out[name] = {"ms_per_launch": ms, "algorithmic_bytes": b,
                     "achieved_gbs": b / (ms * 1e-3) / 1e9, "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm}
    o = out["outer"]
    # assembled 3^d stencil: d^2 FMAs per neighbour block, 3^d blocks per node, + the dot
    flops = 2 * nn * (3 ** p.dim) * p.dim * p.dim + 2 * p.n
    o["algorithmic_flops"] = flops
    o["achieved_gflops"] = flops / (o["ms_per_launch"] * 1e-3) / 1e9
    dom = max(out, key=lambda k: out[k]["ms_per_launch"])
    if dom == "outer":
        head = {"kernel": "k_stencil_apply_dot<%d> (FP64 outer q = K p + p.q)" % p.dim,
                "bound": "alu", "achieved": o["achieved_gflops"] / 1e3,
                "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": o["achieved_gflops"] / FP64_PEAK_GFLOPS,
                "peak_source": "nominal FP64 rate (the measured-peaks file has no FP64 figure)"}
    else:
        k = out[dom]
        head = {"kernel": "k_ebe2<float, %s> (FP32 %s, 2D)" % ("1" if dom == "residual" else "2", dom),
                "bound": "hbm", "achieved": k["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": k["frac_hbm"], "peak_source": src}
    traffic = OUTER_TRAFFIC_BYTES if (dom == "outer" and p.dim == 2 and p.n == 592130) else None
    head.update({"traffic": traffic, "ms_per_launch": out[dom]["ms_per_launch"], "kernels": out})
    return head


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


# the oracle's FP64 PCG (hybrid, cap 1500) reaches 1e-8 here in 125 iterations with the degree-2
# Chebyshev smoother of the headline (211 with one Jacobi sweep; 176 with two GMRES steps per
# smoothing, flexible CG)
ORACLE_ITERATIONS = {"chebyshev": 125, "jacobi": 211, "gmres": 176}


def _cpu_seconds():
    import resource
    r = resource.getrusage(resource.RUSAGE_SELF)
    return r.ru_utime + r.ru_stime


def cpu_baseline(iters=40, warmup=0, steps=1, smoother="chebyshev"):
    """The oracle (plain FP64 numpy / scipy) on the host cores, on a bounded sample of the same
    workload: its hierarchy setup once, then `steps` samples of `iters` PCG iterations.  A solve
    is setup + ORACLE_ITERATIONS iterations at the median per-iteration time.  `cores` is the
    CPU time over the wall time of the sample (the threads BLAS and scipy actually kept busy)."""
    import workloads as W
    from oracle import solve as osolve, mg, krylov, fem

    p = W.cantilever_2d(**WORKLOAD)
    c0, t0 = _cpu_seconds(), time.perf_counter()
    H = osolve.build(p, pc=HEADLINE["pc"], cap=HEADLINE["max_coarse_dofs"],
                     n_geo=HEADLINE["n_geo_levels"], smoother=smoother)
    t_setup = time.perf_counter() - t0
    A0 = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * p.f[0]
    M = lambda v: mg.vcycle(H, v)  # noqa: E731
    for _ in range(warmup):
        krylov.pcg(A0, b, M=M, rtol=0.0, max_iter=1)
    per_it = []
    for _ in range(steps):
        t1 = time.perf_counter()
        krylov.pcg(A0, b, M=M, rtol=0.0, max_iter=iters)
        per_it.append((time.perf_counter() - t1) / iters)
    wall = time.perf_counter() - t0
    cores = (_cpu_seconds() - c0) / wall
    t_it = statistics.median(per_it)
    n_it = ORACLE_ITERATIONS[smoother]
    step_s = t_setup + n_it * t_it
    return {"value": 1.0 / step_s, "unit": "solves/s", "cores": round(cores, 1),
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle hierarchy setup (%.2f s) + %d x %d FP64 PCG iterations (%.1f ms each, "
                      "median; %s smoother) on the full 768x384 workload, scaled to the oracle's "
                      "%d iterations to 1e-8" % (t_setup, steps, iters, 1e3 * t_it, smoother, n_it),
            "ms_per_step": step_s * 1e3, "sample_wall_s": wall}


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only, each step a bounded sample (5 PCG
    iterations) of the same workload, W warm-up iterations first."""
    if rank != 0:
        return None
    cb = cpu_baseline(iters=5, warmup=args.warmup, steps=args.steps, smoother=args.smoother)
    value = cb["value"]
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "2D cantilever quad4 %dx%d (592,130 DOFs), seeded thin 0/1 members "
                       "(1e9 contrast), left edge clamped, unit load right mid-edge"
                       % (WORKLOAD["nx"], WORKLOAD["ny"]),
                       "preconditioner": HEADLINE["pc"], "max_coarse_dofs": HEADLINE["max_coarse_dofs"],
                       "rtol": 1e-8, "smoother": smoother_label(args)},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "host_cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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
        cb = cpu_baseline(smoother=args.smoother)
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "host_cores", "kind",
                                                  "sample")}
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
