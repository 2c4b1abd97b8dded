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
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true")
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
                max_iter=2000, use_graph=args.graph_mode)

    def step(prec):
        u_d.zero_()
        P.set_density(rho_d)
        P.setup(prec=prec, **opts)
        _, res = P.solve(f_d, u0=u_d)
        return res[0]

    def timed(prec, K, Wm):
        for _ in range(Wm):
            step(prec)
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
            r = step(prec)
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
    if args.serving > 0:
        out["serving"] = serving_run(tomg, ctx, args.serving, args.serving_updates, args.slots)
    return out


def serving_run(tomg, ctx, n_requests, n_updates, slots):
    """Replay the mixed 2D/3D request stream (Poisson arrivals, 5 % density noise per update)
    through the continuous-batching server; every update of a request is submitted at the
    request's arrival time and warm-starts from the previous one on the device."""
    import workloads as W
    stream = W.serving_stream(n_requests=n_requests, n_updates=n_updates)
    opt = dict(pc="hybrid", prec="fp32", n_geo_levels=3, max_coarse_dofs=1000, concurrency=1,
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


def roofline(P, ctx, p, stream):
    """Dominant kernel (the level-0 SIMP element operator) timed live with CUDA events on its
    stream; algorithmic bytes per launch from the minimum traffic model."""
    try:
        ms = P.time_fine_operator("apply", "fp32", reps=50, cold_l2=True)
    except Exception as e:  # noqa: BLE001
        return {"error": str(e)}
    peaks = load_peaks()
    nn = (p.nx + 1) * (p.ny + 1)
    # read x, write y (2 x 4 B per DOF), read E once per element, mask byte per node
    bytes_ = 2 * 4 * p.n + 4 * p.nel + nn
    achieved = bytes_ / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"kernel": "ebe_apply fp32 (2D quad4)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "ms_per_launch": ms, "peak_source": "measured" if "fallback" not in peaks else "fallback"}


def cpu_baseline(n_threads_hint=None):
    """Oracle (FP64 numpy/scipy) on the host cores: setup + a bounded number of PCG iterations
    on the same workload, scaled to solves/s with the iteration count the oracle needs."""
    import workloads as W
    from oracle import solve as osolve, mg, krylov, fem

    p = W.cantilever_2d(**WORKLOAD)
    t0 = time.perf_counter()
    H = osolve.build(p, pc=HEADLINE["pc"], cap=HEADLINE["max_coarse_dofs"],
                     n_geo=HEADLINE["n_geo_levels"])
    t_setup = time.perf_counter() - t0
    A0 = mg.fine_operator(p)
    b = fem.free_mask(p.n, p.fixed) * p.f[0]
    k = 10
    t1 = time.perf_counter()
    krylov.pcg(A0, b, M=lambda v: mg.vcycle(H, v), rtol=0.0, max_iter=k)
    t_it = (time.perf_counter() - t1) / k
    return p, H, t_setup, t_it


def run_reference(args, rank, world):
    if rank != 0:
        return None
    p, H, t_setup, t_it = cpu_baseline()
    its_needed = None
    try:
        from oracle import krylov, mg, fem
        its_needed = int(os.environ.get("TOMG_REF_ITERS", "0")) or None
    except Exception:
        pass
    its = its_needed or 210
    step_s = t_setup + its * t_it
    ncores = os.cpu_count()
    value = 1.0 / step_s
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "2D cantilever quad4 %dx%d (592,130 DOFs)" % (WORKLOAD["nx"], WORKLOAD["ny"]),
                       "preconditioner": HEADLINE["pc"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": ncores, "kind": "oracle",
                             "sample": "oracle setup + 10 PCG iterations timed, scaled to %d iterations" % its},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world, local)
        if rank == 0 and not args.no_cpu:
            p, H, t_setup, t_it = cpu_baseline()
            its = out["iterations"]
            step_s = t_setup + its * t_it
            out["cpu_baseline"] = {"value": 1.0 / step_s, "unit": "solves/s", "cores": os.cpu_count(),
                                   "kind": "oracle",
                                   "sample": "oracle hierarchy setup + 10 FP64 PCG iterations on the full "
                                             "workload, scaled to the GPU's %d iterations" % its}
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
