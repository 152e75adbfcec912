"""Benchmark: FMM matvecs/s (and GMRES solves/s) of the Helmholtz single-layer operator.

Default workload: unit sphere, icosphere level 7 + longest-edge bisection
(655,360 triangles x 3 points, N = 1,966,080), k = 20, expansion order
p_l = ceil(k a_l + 6 log10(k a_l + pi)) per level with floor p_min, leaf <= 64,
FP32 P2P/M2L, FP64 GMRES(50) to 1e-4.  One step = one FMM matvec (density prep,
P2P, P2M, M2M, M2L, L2L, L2P, correction, output) with inputs resident in HBM;
the solve (GMRES) is timed in its own region and reported under "solve".

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
Prints ONE JSON line on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvecs/s and solves/s at 1e-4 residual vs plain FP32 form; p50/p99 latency"

WORKLOADS = {
    # name: (mesh, k, config overrides, GMRES restart)
    "sphere_655360": ("sphere_655360", 20.0, {}, 50),
    "sphere_1280": ("sphere_1280", 1.0, {"p_fixed": 8}, 30),
    "sphere_163840": ("sphere_163840", 10.0, {}, 50),
    "sphere_40960": ("sphere_40960", 10.0, {}, 50),
    # GMRES(50) stagnates near 5e-4 on this body at k = 30; GMRES(200) converges
    "ellipsoid_1310720": ("ellipsoid_1310720", 30.0, {}, 200),
    "cap_sphere_387864": ("cap_sphere_387864", 10.0, {}, 50),
}


DRAM_PROFILE = os.path.join(ROOT, "profiles", "dram_sphere_655360.md")
DRAM_WORKLOAD = "sphere_655360"  # the workload that capture ran


def _source_sha(fname):
    import hashlib

    with open(os.path.join(ROOT, "paper_1803_09948_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _ncu_dram(kernel, workload):
    """DRAM bytes (read + write) of one launch of `kernel` on the 1.97 M-point sphere, from the
    committed ncu summary; None on another workload or when the kernel's source file changed
    since the capture."""
    if workload != DRAM_WORKLOAD:
        return None, f"no ncu capture of this workload (the committed one is {DRAM_WORKLOAD})"
    try:
        with open(DRAM_PROFILE) as f:
            kv = dict(line.strip().split(" = ", 1) for line in f if " = " in line and line.startswith("    "))
        files, shas = kv[f"{kernel}.file"].split(","), kv[f"{kernel}.sha256_16"].split(",")
        if any(_source_sha(f_.strip()) != s_.strip() for f_, s_ in zip(files, shas)):
            return None, "kernel changed since the ncu capture"
        return float(kv[f"{kernel}.dram_bytes_per_launch"]), "ncu dram__bytes_read.sum + dram__bytes_write.sum"
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    except Exception:
        return 6800.0, "fallback", 2070.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for q, nm in enumerate(names):
                if r[5 + q].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _max_over_ranks(v, world, device="cuda"):
    """The largest of v over the ranks of the default process group (v itself on one rank)."""
    if world <= 1:
        return float(v)
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank, world, max_ms):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(V, F, k, near_factor, sigma, budget_s=12.0, rows=None):
    """Oracle direct summation on a bounded sample of rows (FP64, all host cores)."""
    import numpy as np

    import oracle

    N = 3 * F.shape[0]
    r = oracle.near_radius(V, F, near_factor)
    rng = np.random.default_rng(1)
    if rows is None:
        probe = rng.choice(N, size=min(16, N), replace=False)
        t0 = time.perf_counter()
        oracle.direct_rows(V, F, k, r, probe, sigma)
        dt = time.perf_counter() - t0
        nrow = int(max(16, min(4096, N, 16 * budget_s / max(dt, 1e-3))))
        rows = np.sort(rng.choice(N, size=nrow, replace=False))
    t0 = time.perf_counter()
    vals = oracle.direct_rows(V, F, k, r, rows, sigma)
    dt = time.perf_counter() - t0
    return rows, vals, dt


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, a bounded sample per step."""
    import numpy as np

    import synthetic

    world, rank, _ = _dist()
    if rank != 0:
        return
    mesh, k, over, _ = WORKLOADS[args.workload]
    V, F = synthetic.workload_mesh(mesh)
    N = 3 * F.shape[0]
    sigma = synthetic.random_density(N, seed=0)
    # size each step so the whole run stays within a few minutes
    rows, _, dt = cpu_baseline(V, F, k, 1.0, sigma, budget_s=min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(V, F, k, 1.0, sigma, rows=rows)
    times = []
    for _ in range(args.steps):
        _, _, dt = cpu_baseline(V, F, k, 1.0, sigma, rows=rows)
        times.append(dt)
    tot = sum(times)
    value = args.steps * len(rows) / N / tot
    sample = f"{len(rows)} sampled rows of the direct sum (point part + exact self/near integrals) per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "k": k},
        "cpu_baseline": {"value": value, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_refine(args):
    """Mixed-precision refinement: inner GMRES on the fast plan (FP32 near field, BF16x3 tensor-core
    M2L, default orders, tolerance 1e-4), outer residuals b - A x in double-float with an accurate plan
    (orders >= refine-pmin, FP32 SIMT M2L, FP64 near field and correction), to 1e-6; plain GMRES to
    1e-4 on the fast plan beside it.  The CPU-baseline leg evaluates both operators' error against
    the oracle's FP64 direct sum on sampled rows."""
    import numpy as np
    import torch

    import __graft_entry__
    import paper_1803_09948_gb300 as pkg
    import synthetic

    if _dist()[1] != 0:  # a single-GPU arm: under torchrun rank 0 runs it, the others exit
        return
    torch.cuda.set_device(0)
    __graft_entry__.build()
    name = args.workload if args.workload != "sphere_655360" else "ellipsoid_1310720"
    mesh, k, over, restart = WORKLOADS[name]
    if args.restart > 0:
        restart = args.restart
    V, F = synthetic.workload_mesh(mesh)
    t0 = time.perf_counter()
    if args.adaptive:
        over = dict(over, adaptive=1)
    if args.leaf_max > 0:
        over = dict(over, leaf_max=args.leaf_max)
    inner = pkg.Plan(V, F, k, restart=restart, tol=1e-4, **over)
    torch.cuda.synchronize()
    t_in = time.perf_counter() - t0
    t0 = time.perf_counter()
    outer = pkg.Plan(V, F, k, p_min=args.refine_pmin, m2l_tensor=0, precision=1, **over)
    torch.cuda.synchronize()
    t_out = time.perf_counter() - t0
    N = inner.n
    b = torch.empty(N, dtype=torch.complex64, device="cuda")
    inner.rhs_planewave([0.0, 0.0, 1.0], b)
    x = torch.empty_like(b)
    xp = torch.empty_like(b)
    clocks = ClockSampler(0)
    clocks.start()
    inner.solve(b, xp)  # warm-up (Krylov basis)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sp, itp, rrp = inner.solve(b, xp)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    st, nout, nin, rr = inner.solve_refined(outer, b, x, tol=1e-6, max_outer=10)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    clk = clocks.stop()
    # the plain solution's residual under the accurate operator, for comparison
    y = torch.empty_like(b)
    outer.matvec(xp, y)
    torch.cuda.synchronize()
    bb = b.cpu().numpy().astype(np.complex128)
    res_plain_outer = float(np.linalg.norm(bb - y.cpu().numpy()) / np.linalg.norm(bb))
    d = torch.from_numpy(synthetic.random_density(N, 0).astype(np.complex64)).cuda()
    o = torch.empty_like(d)
    inner.matvec(d, o)
    stages_in = inner.matvec_timed(d, o)
    outer.matvec(d, o)
    stages_out = outer.matvec_timed(d, o)
    # ------------------------------------------------ operator errors and CPU baseline (oracle rows)
    op_err, cpu = None, None
    if not args.no_cpu_baseline:
        s = synthetic.random_density(N, 7).astype(np.complex128)
        od = torch.empty(N, 4, dtype=torch.float32, device="cuda")
        outer.matvec_df(pkg.df_from_complex(s), od)
        s32 = torch.from_numpy(s.astype(np.complex64)).cuda()
        o32 = torch.empty_like(s32)
        inner.matvec(s32, o32)
        torch.cuda.synchronize()
        got_out, got_in = pkg.df_to_complex(od), o32.cpu().numpy().astype(np.complex128)
        rows, ref, dt = cpu_baseline(V, F, k, outer.cfg.near_factor, s, budget_s=20.0)
        nref = np.linalg.norm(ref)
        op_err = {"sampled_rows": int(len(rows)), "outer_rel_err": float(np.linalg.norm(got_out[rows] - ref) / nref),
                  "inner_rel_err": float(np.linalg.norm(got_in[rows] - ref) / nref),
                  "note": "random density; outer in double-float (hfmm_matvec_df), inner complex64"}
        cpu = {"value": len(rows) / N / dt, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(rows)} sampled rows of the FP64 direct sum, {dt:.1f} s, scaled to whole matvecs"}
    print(json.dumps({
        "metric": METRIC, "value": 1.0 / t_ref, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32 FMM (inner BF16x3 tensor-core M2L); fp64-class refinement residual and Arnoldi",
        "data": "synthetic",
        "config": {"workload": f"{name}: {synthetic.WORKLOADS[mesh][0]}", "N": N, "k": k,
                   "inner": {"orders": inner.info()["orders"], "m2l": "tcgen05 BF16x3 where (p+1)^2 <= 64",
                             "restart": restart, "tol": 1e-4},
                   "outer": {"orders": outer.info()["orders"], "m2l": "FP32 SIMT",
                             "near_field_and_correction": "FP64 (precision = 1)"}},
        "refined": {"status": "converged" if st == 0 else "not converged", "relres_outer_operator": rr,
                    "outer_steps": nout, "inner_gmres_iterations": nin, "seconds": t_ref},
        "plain": {"status": "converged" if sp == 0 else "not converged", "relres": rrp[0], "iterations": itp[0],
                  "seconds": t_plain, "relres_outer_operator": res_plain_outer},
        "plan_s": {"inner": t_in, "outer": t_out},
        "matvec_ms": {"inner": sum(stages_in.values()), "outer": sum(stages_out.values())},
        "device_bytes": {"inner": inner.info()["device_bytes"], "outer": outer.info()["device_bytes"]},
        "operator_error_vs_oracle": op_err,
        "cpu_baseline": cpu,
        "clocks": clk,
    }))
    inner.close()
    outer.close()


def run_serving(args):
    """Serving: seeded requests with Poisson arrivals (20 per second), sphere / ellipsoid /
    star geodesic meshes with N log-uniform in [10k, serve-nmax], k uniform in
    [1, serve-kmax], 1..16 right-hand sides; admitted by an 80 % device-memory budget."""
    import numpy as np
    import torch

    import __graft_entry__
    import synthetic
    from paper_1803_09948_gb300 import serving

    if _dist()[1] != 0:  # a single-GPU arm: under torchrun rank 0 runs it, the others exit
        return
    torch.cuda.set_device(0)
    __graft_entry__.build()
    specs = synthetic.serving_requests(args.serve, seed=0, rate=20.0, n_max=args.serve_nmax,
                                       k_range=(1.0, args.serve_kmax))
    reqs = []
    for sp in specs:  # meshes come with the requests: built before the clock starts
        V, F = synthetic.serving_shape(sp["shape"], sp["nu"], sp["seed"])
        dirs = np.asarray(synthetic.fibonacci_directions(sp["nrhs"], seed=sp["seed"] % 100000)).reshape(-1, 3)
        reqs.append(dict(sp, V=V, F=F, dirs=dirs))
    eng = serving.ServingEngine(max_inflight=args.serve_slots, restart=30, tol=1e-4, max_iter=args.serve_maxiter,
                                group_max=args.serve_group)
    clocks = ClockSampler(0)
    clocks.start()
    records, summ = eng.run(reqs)
    clk = clocks.stop()
    print(json.dumps({
        "metric": METRIC, "value": summ["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32 (P2P, M2L, tree passes); fp64-class GMRES", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} requests, Poisson arrivals 20/s, sphere / ellipsoid (2,1,1) / "
                               f"star geodesic meshes, N log-uniform in [10k, {args.serve_nmax}], k uniform in "
                               f"[1, {args.serve_kmax}], 1-16 plane-wave right-hand sides, GMRES(30) to 1e-4 "
                               f"(at most {args.serve_maxiter} iterations)",
                   "slots": args.serve_slots, "budget": "80% of device memory (admission by memory, in arrival order)",
                   "groups": "single-RHS requests of <= 200k points arriving within 50 ms: up to 8 per group solve, "
                             "one shared graph launch per restart cycle" if args.serve_group > 1 else "off"},
        "latency_s": {"p50": summ["latency_p50_s"], "p99": summ["latency_p99_s"], "mean": summ["latency_mean_s"]},
        "serving": summ,
        "requests": [dict({k_: r.get(k_) for k_ in ("id", "n_points", "nrhs", "status", "latency_s", "wait_s",
                                                    "build_s", "solve_s", "iterations", "error",
                                                    "estimate_bytes", "device_bytes", "group_size")},
                          k=next(q["k"] for q in reqs if q["id"] == r["id"]), shape=next(q["shape"] for q in reqs if q["id"] == r["id"]))
                     for r in sorted(records, key=lambda r: r["id"])],
        "clocks": clk,
    }))


def run_batched(args):
    """Batched right-hand sides: one step = one matvec of args.nrhs plane-wave right-hand sides
    (seeded Fibonacci directions), all in one captured CUDA graph; value counts right-hand sides."""
    import numpy as np
    import torch

    import __graft_entry__
    import paper_1803_09948_gb300 as pkg
    import synthetic

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    __graft_entry__.build()
    mesh, k, over, restart = WORKLOADS[args.workload]
    cfg = dict(over)
    if args.simt:
        cfg["m2l_tensor"] = 0
    if args.adaptive:
        cfg["adaptive"] = 1
    if args.leaf_max > 0:
        cfg["leaf_max"] = args.leaf_max
    for key in ("p2p_kernel", "m2l_kernel", "overlap", "tc_group", "autotune"):
        if getattr(args, key) is not None:
            cfg[key] = getattr(args, key)
    V, F = synthetic.workload_mesh(mesh)
    N, R = 3 * F.shape[0], args.nrhs
    stream = torch.cuda.current_stream()
    plan = pkg.Plan(V, F, k, **cfg)
    info = plan.info()
    dirs = np.asarray(synthetic.fibonacci_directions(R, seed=0)).reshape(R, 3)
    b = torch.empty(R * N, dtype=torch.complex64, device="cuda")
    plan.rhs_planewave(dirs, b)
    out = torch.empty_like(b)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        plan.matvec(b, out, R)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = plan.launch_count()
    barrier()
    ev[0].record(stream)
    for s_ in range(args.steps):
        plan.matvec(b, out, R)
        ev[s_ + 1].record(stream)
    barrier()
    launches = plan.launch_count() - launches0
    clk = clocks.stop()
    step_ms = [ev[q].elapsed_time(ev[q + 1]) for q in range(args.steps)]
    total_ms = _max_over_ranks(ev[0].elapsed_time(ev[args.steps]), world)
    value = _job_rate(args.steps * R, world, total_ms)
    # the same right-hand sides one at a time (context: the plain single right-hand-side form)
    b1, o1 = b[:N].clone(), torch.empty(N, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        plan.matvec(b1, o1, 1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        plan.matvec(b1, o1, 1)
    e1.record(stream)
    barrier()
    single_ms = e0.elapsed_time(e1) / 10
    # end to end: right-hand sides from pinned host memory and potentials back, every step
    h_in = b.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    for _ in range(2):
        b.copy_(h_in, non_blocking=True)
        plan.matvec(b, out, R)
        h_out.copy_(out, non_blocking=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        b.copy_(h_in, non_blocking=True)
        plan.matvec(b, out, R)
        h_out.copy_(out, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1), world)
    got = h_out.numpy().astype(np.complex128).reshape(R, N)
    S = h_in.numpy().astype(np.complex128).reshape(R, N)
    # R solves in lockstep (GMRES per right-hand side on shared batched matvecs), own timed region
    solve = None
    if args.solves > 0:
        xs = torch.empty_like(b)
        plan.solve(b, xs, R)  # warm-up (allocates the Krylov bases)
        lat, its_all, rr_all = [], None, None
        for _ in range(args.solves):
            barrier()
            t1 = time.perf_counter()
            stt, its_all, rr_all = plan.solve(b, xs, R)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t1)
        x1 = torch.empty(N, dtype=torch.complex64, device="cuda")
        plan.solve(b1, x1)
        barrier()
        t1 = time.perf_counter()
        plan.solve(b1, x1)
        torch.cuda.synchronize()
        single_solve_ms = 1e3 * (time.perf_counter() - t1)
        solve = {"solves_per_s": R * len(lat) / sum(lat), "ms_per_batch": 1e3 * statistics.mean(lat),
                 "single_rhs_solve_ms": single_solve_ms,
                 "nrhs": R, "iterations_max": int(max(its_all)), "iterations_min": int(min(its_all)),
                 "true_relres_max": float(max(rr_all)), "restart": restart, "tol": 1e-4,
                 "status": "converged" if stt == 0 else "not converged",
                 "rhs": f"{R} plane waves (seeded Fibonacci directions)"}
    acc, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        picks = sorted({0, R // 3, (2 * R) // 3, R - 1})
        errs, rows_n, t_cpu = [], 0, 0.0
        for r in picks:
            rows, ref, dt = cpu_baseline(V, F, k, plan.cfg.near_factor, S[r], budget_s=4.0)
            errs.append(float(np.linalg.norm(got[r][rows] - ref) / np.linalg.norm(ref)))
            rows_n, t_cpu = rows_n + len(rows), t_cpu + dt
        acc = {"rhs_checked": picks, "sampled_rows_each": rows_n // len(picks), "rel_err_vs_oracle": errs,
               "max_rel_err": max(errs)}
        cpu = {"value": rows_n / N / t_cpu, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{rows_n} sampled rows over {len(picks)} right-hand sides of the FP64 direct sum "
                         f"(point part + exact self/near integrals), {t_cpu:.1f} s, scaled to whole matvecs"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32 (P2P, M2L, tree passes)", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {synthetic.WORKLOADS[mesh][0]}, {R} plane-wave right-hand "
                                   "sides (seeded Fibonacci directions) per batched matvec",
                       "N": N, "k": k, "nrhs": R, "orders": info["orders"], "graph": "one captured CUDA graph per step",
                       "kernels": plan.tuning(), "autotune": plan.cfg.autotune,
                       "m2l": "FP32 SIMT" if args.simt else "tcgen05 BF16x3 (levels with (p+1)^2 <= 64), FP32 SIMT above",
                       "l2": "inputs larger than L2 (batched expansions alone exceed it)"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "mean": statistics.mean(step_ms)},
            "solve": solve,
            "single_rhs_ms": single_ms,
            "speedup_per_rhs_vs_single": single_ms / (total_ms / args.steps / R),
            "e2e": {"value": _job_rate(args.steps * R, world, e2e_ms), "unit": "matvec/s", "h2d_bytes_per_step": 8 * N * R,
                    "d2h_bytes_per_step": 8 * N * R},
            "roofline": None,
            "cpu_baseline": cpu,
            "accuracy": acc,
            "clocks": clk,
            "gpu_launches": launches,
        }))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="sphere_655360", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--p-min", type=int, default=None)
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--plain-steps", type=int, default=20,
                    help="matvecs of the plain single-RHS FP32 form (SIMT M2L) timed beside the headline; 0: skip")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--simt", action="store_true", help="M2L on FP32 SIMT cores only (the plain form)")
    ap.add_argument("--leaf-max", type=int, default=0, help="> 0: points per leaf at most (default: the plan's 64)")
    ap.add_argument("--adaptive", action="store_true",
                    help="adaptive octree (boxes split only above leaf_max points; leaves at several depths)")
    ap.add_argument("--refine", action="store_true",
                    help="mixed-precision refinement to 1e-6 beside plain GMRES to 1e-4 (default workload: the ellipsoid)")
    ap.add_argument("--refine-pmin", type=int, default=12, help="minimum order of the outer (residual) plan")
    ap.add_argument("--restart", type=int, default=0, help="> 0: GMRES restart length instead of the workload's")
    ap.add_argument("--p2p-kernel", type=int, default=None, help="near-field kernel (0 staged, 1 packed)")
    ap.add_argument("--overlap", type=int, default=None, help="1: two-branch captured matvec, 0: sequential")
    ap.add_argument("--m2l-kernel", type=int, default=None,
                    help="tensor-core M2L (0 source-stationary items, 1 target-stationary tiles)")
    ap.add_argument("--tc-group", type=int, default=None, help="work items per tensor-core block (8, 16, 32)")
    ap.add_argument("--autotune", type=int, default=None, help="1: tune the kernel choices at plan creation")
    ap.add_argument("--serve", type=int, default=0, help="> 0: serving workload with this many requests")
    ap.add_argument("--serve-nmax", type=int, default=1_000_000)
    ap.add_argument("--serve-kmax", type=float, default=30.0)
    ap.add_argument("--serve-slots", type=int, default=64, help="most requests in flight (memory admits first)")
    ap.add_argument("--serve-maxiter", type=int, default=300, help="GMRES iteration cap per request")
    ap.add_argument("--serve-group", type=int, default=8, help="most single-RHS requests per group solve (1: off)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="> 1: batched plane-wave right-hand sides in one graph-captured matvec per step")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.nrhs > 1:
        return run_batched(args)
    if args.serve > 0:
        return run_serving(args)
    if args.refine:
        return run_refine(args)

    import numpy as np
    import torch

    import __graft_entry__
    import paper_1803_09948_gb300 as pkg
    import synthetic

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    __graft_entry__.build()
    mesh, k, over, restart = WORKLOADS[args.workload]
    cfg = dict(over)
    if args.p_min is not None:
        cfg["p_min"] = args.p_min
    cfg["restart"] = restart
    if args.simt:
        cfg["m2l_tensor"] = 0
    if args.adaptive:
        cfg["adaptive"] = 1
    if args.leaf_max > 0:
        cfg["leaf_max"] = args.leaf_max
    for key in ("p2p_kernel", "m2l_kernel", "overlap", "tc_group", "autotune"):
        if getattr(args, key) is not None:
            cfg[key] = getattr(args, key)
    V, F = synthetic.workload_mesh(mesh)
    N = 3 * F.shape[0]
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = pkg.Plan(V, F, k, **cfg)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    costs = plan.costs()
    sigma = synthetic.random_density(N, seed=0)
    dens = torch.from_numpy(sigma.astype(np.complex64)).cuda()
    pot = torch.empty_like(dens)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ------------------------------------------------------------ device-resident matvecs
    for _ in range(args.warmup):
        plan.matvec(dens, pot)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = plan.launch_count()
    barrier()
    ev[0].record(stream)
    for s in range(args.steps):
        plan.matvec(dens, pot)
        ev[s + 1].record(stream)
    barrier()
    launches = plan.launch_count() - launches0
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = _max_over_ranks(ev[0].elapsed_time(ev[args.steps]), world)
    clk = clocks.stop()
    value = _job_rate(args.steps, world, total_ms)

    # ------------------------------------------------------------ per-stage breakdown (same stream)
    stages = None
    reps = 3
    for r in range(reps):
        st = plan.matvec_timed(dens, pot)
        stages = st if stages is None else {q: stages[q] + st[q] for q in st}
    stages = {q: v / reps for q, v in stages.items()}

    # ------------------------------------------------------------ end to end through the ABI (host buffers)
    # hfmm_matvec_host: density copied in from page-locked host memory, potential copied back,
    # inside the call, every step
    h_in = torch.from_numpy(sigma.astype(np.complex64)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    for _ in range(2):
        plan.matvec_host(h_in, h_out)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.matvec_host(h_in, h_out)
    e1.record(stream)
    barrier()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1), world)
    got = h_out.numpy().astype(np.complex128)

    # ------------------------------------------------------------ GMRES solves (own region)
    solve = None
    if args.solves > 0:
        b = torch.empty_like(dens)
        plan.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(dens)
        plan.solve(b, x)  # warm-up solve (allocates the Krylov basis)
        lat = []
        its = []
        rrs = []
        for _ in range(args.solves):
            barrier()
            t1 = time.perf_counter()
            stt, it, rr = plan.solve(b, x)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t1)
            its.append(it[0])
            rrs.append(rr[0])
        solve = {"solves_per_s": len(lat) / sum(lat), "ms_per_solve": 1e3 * statistics.mean(lat),
                 "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "iterations": its[-1], "true_relres": rrs[-1], "restart": restart, "tol": 1e-4,
                 "status": "converged" if stt == 0 else "not converged", "rhs": "plane wave along +z"}
        # everything but the matvecs (one per iteration and one true residual per restart cycle),
        # per Arnoldi step: orthogonalisation, norms, Hessenberg bookkeeping, launches, the
        # per-iteration 16-byte read of the residual estimate
        n_mv = its[-1] + -(-its[-1] // restart)
        solve["arnoldi_ms_per_step"] = (solve["ms_per_solve"] - n_mv * total_ms / args.steps) / max(its[-1], 1)

    # ------------------------------------------------------------ the plain single-RHS FP32 form
    # (M2L on FP32 SIMT at every level), same workload, same CUDA-event timing on the same stream
    plain = None
    if not args.simt and args.plain_steps > 0:
        pplan = pkg.Plan(V, F, k, **dict(cfg, m2l_tensor=0))
        ppot = torch.empty_like(dens)
        for _ in range(args.warmup):
            pplan.matvec(dens, ppot)
        barrier()
        e0.record(stream)
        for _ in range(args.plain_steps):
            pplan.matvec(dens, ppot)
        e1.record(stream)
        barrier()
        plain_ms = _max_over_ranks(e0.elapsed_time(e1), world) / args.plain_steps
        pstages = pplan.matvec_timed(dens, ppot)
        pgot = ppot.cpu().numpy().astype(np.complex128)
        plain = {"value": _job_rate(1, world, plain_ms), "unit": "matvec/s", "ms_per_matvec": plain_ms,
                 "steps": args.plain_steps, "m2l": "FP32 SIMT at every level", "stages_ms": pstages,
                 "speedup_of_headline": plain_ms / (total_ms / args.steps)}
        if args.solves > 0:
            b = torch.empty_like(dens)
            pplan.rhs_planewave([0.0, 0.0, 1.0], b)
            x2 = torch.empty_like(dens)
            pplan.solve(b, x2)  # warm-up (Krylov basis)
            barrier()
            t1 = time.perf_counter()
            stt2, it2, rr2 = pplan.solve(b, x2)
            torch.cuda.synchronize()
            plain["solve"] = {"ms_per_solve": 1e3 * (time.perf_counter() - t1), "iterations": it2[0],
                              "true_relres": rr2[0], "status": "converged" if stt2 == 0 else "not converged"}
        pplan.close()

    # ------------------------------------------------------------ roofline of the dominant stage
    hbm, peak_src, smax = _peaks()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = json.load(f).get("bf16_tflops", 1936.2)
    except Exception:
        bf16_peak = 1900.0
    props = torch.cuda.get_device_properties(local)
    fp32_peak = props.multi_processor_count * 128 * 2 * smax * 1e6 / 1e12  # TFLOP/s
    dom = max(stages, key=stages.get)
    tc_cmacs = costs["m2l_tc_cmacs"]
    tuning = plan.tuning()
    # stage -> (bound, algorithmic amount per launch, unit, peak, convention, kernel name for ncu)
    work = {
        "p2p": ("alu", costs["p2p_pairs"] * 24 / 1e12, "TFLOP/s", fp32_peak, "24 flop per source-target pair",
                "k_p2p_packed" if tuning["p2p_kernel"]["choice"] == 1 else "k_p2p_staged"),
        "m2l_simt": ("alu", (costs["m2l_cmacs"] - tc_cmacs) * 8 / 1e12, "TFLOP/s", fp32_peak,
                     "8 flop per complex multiply-add, P_l^2 per translation (SIMT levels)", None),
        "m2l": ("tensor", tc_cmacs * 8 / 1e12, "TFLOP/s", bf16_peak,
                "the method's flops: 8 per complex multiply-add, P^2 per translation "
                f"({int(costs['m2l_tc_translations'])} translations per launch)",
                "k_m2l_ts" if tuning["m2l_kernel"]["choice"] == 1 else "k_m2l_tc"),
        "corr": ("hbm", (costs["corr_nnz"] * 12 + costs["n_points"] * 16) / 1e9, "GB/s", hbm,
                 "12 B per nonzero + 16 B per row", "k_corr"),
    }
    peak_source = {"alu": f"FP32: {props.multi_processor_count} SMs x 128 lanes x 2 flop x {smax:.0f} MHz",
                   "tensor": f"dense BF16 cuBLAS burst, {peak_src}", "hbm": f"HBM {peak_src} copy bandwidth"}

    def _roof(stage):
        bound, amount, unit, peak, note, kname = work[stage]
        achieved = amount / (stages[stage] / 1e3)
        traffic, tnote = _ncu_dram(kname, args.workload) if kname else (None, "no ncu capture")
        return {"kernel": kname or stage, "stage": stage, "bound": bound, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": traffic, "traffic_source": tnote,
                "peak_source": peak_source[bound], "work_per_launch": note}

    rl = _roof(dom) if dom in work else None
    if rl is not None and dom == "m2l":
        # what the tensor pipe executes: each multiply-add as three BF16 products (hi*hi, hi*lo, lo*hi)
        rl["issued_bf16x3"] = {"achieved": 3 * rl["achieved"], "frac": 3 * rl["achieved"] / bf16_peak,
                               "note": "three BF16 products per multiply-add of the split; the method's work is "
                                       "a third of it (frac above)"}
    p2p_block = _roof("p2p")
    # tree passes: bytes by the stated model (8 B per complex coefficient, 16 B per point
    # position, 8 B per density / potential value), against the measured HBM copy bandwidth
    nL, c_leaf = costs["n_points"], costs["leaf_coefficients"]
    c_all, c2, cL = costs["multipole_coefficients"], costs["level2_coefficients"], costs["levelL_coefficients"]
    tree_model = {
        "p2m": ("k_p2m_w", nL * (16 + 8) + 8 * c_leaf, "read points and densities, write leaf multipoles"),
        "m2m": ("m2m", 8 * (2 * c_all - c2 - cL), "read children's multipoles, write parents'"),
        "l2l": ("l2l", 8 * (2 * c_all - c2 - cL), "read parents' locals, add into children's"),
        "l2p": ("k_l2p_t", nL * (16 + 8 + 8) + 8 * c_leaf, "read points, leaf locals and potentials, write potentials"),
    }
    tree = {}
    for stg, (kname, nbytes, note) in tree_model.items():
        gbs = nbytes / 1e9 / (stages[stg] / 1e3)
        traffic, tnote = _ncu_dram(kname, args.workload)
        tree[stg] = {"ms": stages[stg], "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm,
                     "model": note, "traffic": traffic, "traffic_source": tnote,
                     "dram_gbs": traffic / 1e9 / (stages[stg] / 1e3) if traffic else None}

    # ------------------------------------------------------------ accuracy and CPU baseline (rank 0)
    cpu = None
    acc = None
    if rank == 0 and not args.no_cpu_baseline:
        rows, ref, dt = cpu_baseline(V, F, k, plan.cfg.near_factor, sigma)
        acc = {"sampled_rows": int(len(rows)),
               "rel_err_vs_oracle": float(np.linalg.norm(got[rows] - ref) / np.linalg.norm(ref))}
        if plain is not None:
            plain["rel_err_vs_oracle"] = float(np.linalg.norm(pgot[rows] - ref) / np.linalg.norm(ref))
        cpu = {"value": len(rows) / N / dt, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(rows)} sampled rows of the FP64 direct sum (point part + exact self/near "
                         f"integrals), {dt:.1f} s, scaled to whole matvecs"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("fp32 (P2P, tree passes, M2L on every level)" if args.simt else
                      "fp32 (P2P, tree passes, SIMT M2L at (p+1)^2 > 64); bf16x3 split with fp32 accumulation "
                      "(tensor-core M2L at (p+1)^2 <= 64)") + "; fp64-class double-float GMRES",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {synthetic.WORKLOADS[mesh][0]}", "N": N, "k": k,
                       "leaf_max": plan.cfg.leaf_max, "depth": info["depth"], "orders": info["orders"],
                       "near_factor": plan.cfg.near_factor, "corr_nnz": info["corr_nnz"],
                       "m2l": "FP32 SIMT" if args.simt else "tcgen05 BF16x3 (levels with (p+1)^2 <= 64), FP32 SIMT above",
                       "m2l_translations": info["m2l_translations"], "device_bytes": info["device_bytes"],
                       "tree": "adaptive" if args.adaptive else "uniform", "leaves": info["n_leaves"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 (plan holds {info['device_bytes'] / 1e9:.2f} GB)",
                       "kernels": tuning, "autotune": plan.cfg.autotune},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "mean": statistics.mean(step_ms),
                           "std": statistics.pstdev(step_ms) if len(step_ms) > 1 else 0.0},
            "stages_ms": stages,
            "plan_s": plan_s,
            "solve": solve,
            "e2e": {"value": _job_rate(args.steps, world, e2e_ms), "unit": "matvec/s", "h2d_bytes_per_step": 8 * N,
                    "d2h_bytes_per_step": 8 * N},
            "roofline": rl,
            "p2p": p2p_block,
            "tree_passes": tree,
            "plain_fp32": plain,
            "cpu_baseline": cpu,
            "accuracy": acc,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(out))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
