"""Serving loop for scattering solves.

Requests (a surface mesh, a wavenumber k and one or more incident directions)
arrive over time; each is solved with the FMM-accelerated GMRES of the library:
its plan (octree, translation operators, near-field correction) and Krylov
basis are built on the device when the request is admitted, stay resident
until its solve has finished, and are then released.

  * Admission: a request is started as soon as the device memory reserved by
    the requests in flight, plus its own estimate, stays within the budget
    (by default 80 % of the device's memory) and a slot is free; requests are
    admitted in arrival order.  A request whose estimate alone exceeds the
    budget is rejected.
  * Concurrency: every admitted request runs at once on its own host thread and
    CUDA stream (up to `max_inflight` slots, 64 by default, so that the memory
    budget is what bounds it), so the plan building of some requests (host
    octree and lists, device operator and correction kernels) overlaps the
    solves of others and their kernels share the device.
  * Shared launches: single right-hand-side requests of at most `group_n_max`
    points (200k) that arrive within `group_wait_s` (50 ms) of the first of them
    are served as one group (up to `group_max`, 8): their plans are built side
    by side, then hfmm_solve_group advances all their GMRES solves together,
    every restart cycle of all unfinished solves inside one graph launch (a
    gated while node per solve).  Requests keep their own admission (memory,
    slot) and records.
  * Multi-RHS requests use the library's lockstep solver (one batched,
    graph-captured matvec per GMRES iteration for all directions).

Latency of a request = completion (its solution copied back to the host)
minus arrival. `ServingEngine.run` returns per-request records and a summary
with p50 / p99 latency and solves per second (right-hand sides solved per
second of wall time from the first arrival to the last completion).
"""
from __future__ import annotations

import threading
import time

import numpy as np


def _order(k: float, a: float, p_min: int = 7) -> int:
    """The plan's per-level expansion order p = ceil(k a + 6 log10(k a + pi)), at least p_min."""
    import math

    return max(p_min, int(math.ceil(k * a + 6.0 * math.log10(k * a + math.pi))))


def estimate_bytes(n_points: int, nrhs: int, restart: int, k: float = 0.0, extent: float = 0.0,
                   leaf_max: int = 64) -> int:
    """Device memory of one request: plan (about 1.2 KB per point: sorted points, the
    near-field correction, expansions) plus its translation operators (per level from 2 to
    the leaf level: 316 M2L matrices of (p+1)^2 x (p+1)^2 complex64 and 16 M2M / L2L ones,
    p from the plan's order formula on a box of side extent / 2^l), plus the Krylov basis and
    work vectors ((restart + 1) + 4 double-float vectors per right-hand side, 16 B per point
    each) plus, for several right-hand sides, the batched matvec buffers; 128 MB of slack."""
    import math

    per_point = 1200 + 16 * nrhs * (restart + 5)
    if nrhs > 1:
        per_point += 200 * nrhs
    ops = 0
    if k > 0.0 and extent > 0.0:
        depth = max(2, int(math.ceil(math.log(max(n_points / leaf_max, 1.0)) / math.log(4.0))) + 1)
        prev = None
        for lev in range(2, depth + 1):
            a = 0.5 * math.sqrt(3.0) * extent / 2 ** lev
            P = (_order(k, a) + 1) ** 2
            ops += 316 * P * P * 8 + (16 * P * prev * 8 if prev else 0)
            prev = P
    return int(n_points * per_point + ops + (128 << 20))


class Admission:
    """Device-memory budget shared by the workers; grants in request order."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.in_use = 0
        self.peak = 0
        self._cv = threading.Condition()
        self._next = 0  # ticket served next (FIFO among waiting requests)
        self._tickets = 0

    def ticket(self) -> int:
        with self._cv:
            t = self._tickets
            self._tickets += 1
            return t

    def acquire(self, ticket: int, nbytes: int) -> bool:
        """Blocks until it is this ticket's turn and nbytes fit; False if they never can."""
        with self._cv:
            while ticket != self._next:
                self._cv.wait()
            if nbytes > self.budget:
                self._next += 1
                self._cv.notify_all()
                return False
            while self.in_use + nbytes > self.budget:
                self._cv.wait()
            self.in_use += nbytes
            self.peak = max(self.peak, self.in_use)
            self._next += 1
            self._cv.notify_all()
            return True

    def release(self, nbytes: int):
        with self._cv:
            self.in_use -= nbytes
            self._cv.notify_all()


def gpu_executor(restart: int = 30, tol: float = 1e-4, keep_solution: bool = False, max_iter: int = 1000,
                 max_building: int = 8):
    """Executor that solves a request with the library on the calling thread's stream.
    Returns a function(request, stream) -> dict of timings and results (with the
    solutions, [nrhs][N] complex64 on the host, under "x" when keep_solution)."""
    import torch

    from . import Plan

    # at most max_building plans are built at once: a build is mostly host work (octree, lists,
    # work items) plus short device kernels, and dozens at once only slow every one of them down
    building = threading.Semaphore(max_building)

    def run(req, stream):
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            with building:
                plan = Plan(req["V"], req["F"], req["k"], stream=stream, restart=restart, tol=tol, max_iter=max_iter)
                stream.synchronize()  # plan ready (its build is part of the request's time); only this
                # request's stream: a device-wide wait would stall every other request in flight
            try:
                t1 = time.perf_counter()
                R, N = req["nrhs"], plan.n
                b = torch.empty(R * N, dtype=torch.complex64, device="cuda")
                plan.rhs_planewave(np.asarray(req["dirs"]).reshape(R, 3), b, stream=stream)
                x = torch.empty_like(b)
                status, its, rr = plan.solve(b, x, R, stream=stream)
                x_host = x.to("cpu", non_blocking=False)  # the response
                t2 = time.perf_counter()
                out = {"status": int(status), "iterations": [int(v) for v in its],
                       "relres": [float(v) for v in rr], "n_points": N, "build_s": t1 - t0,
                       "solve_s": t2 - t1, "device_bytes": plan.info()["device_bytes"],
                       "response_bytes": x_host.numel() * 8}
                if keep_solution:
                    out["x"] = x_host.numpy().reshape(R, N)
                return out
            finally:
                plan.close()

    return run


def gpu_group_executor(restart: int = 30, tol: float = 1e-4, keep_solution: bool = False, max_iter: int = 1000,
                       max_building: int = 8):
    """Executor for a group of single right-hand-side requests: their plans are built (at most
    max_building at once), then hfmm_solve_group advances all their GMRES solves together, each
    restart cycle of every unfinished solve inside one shared graph launch.  Returns a function
    (requests, stream) -> list of per-request dicts (as gpu_executor's)."""
    import concurrent.futures as cf

    import torch

    from . import Plan, hfmm_solve_group

    def run(reqs, stream):
        t0 = time.perf_counter()
        plans = [None] * len(reqs)
        build_s = [0.0] * len(reqs)

        def build(q):
            t = time.perf_counter()
            with torch.cuda.stream(stream):
                plans[q] = Plan(reqs[q]["V"], reqs[q]["F"], reqs[q]["k"], stream=stream, restart=restart, tol=tol,
                                max_iter=max_iter)
            build_s[q] = time.perf_counter() - t

        try:
            with cf.ThreadPoolExecutor(max_workers=max(1, min(max_building, len(reqs)))) as ex:
                list(ex.map(build, range(len(reqs))))
            stream.synchronize()
            t1 = time.perf_counter()
            with torch.cuda.stream(stream):
                bs, xs = [], []
                for p, r in zip(plans, reqs):
                    b = torch.empty(p.n, dtype=torch.complex64, device="cuda")
                    p.rhs_planewave(np.asarray(r["dirs"]).reshape(1, 3), b, stream=stream)
                    bs.append(b)
                    xs.append(torch.empty_like(b))
                status, its, rrs = hfmm_solve_group(plans, bs, xs, stream=stream)
                hosts = [x.to("cpu", non_blocking=False) for x in xs]
            t2 = time.perf_counter()
            outs = []
            for q, (p, r) in enumerate(zip(plans, reqs)):
                ok = rrs[q] <= tol
                o = {"status": 0 if ok else 1, "iterations": [int(its[q])], "relres": [float(rrs[q])],
                     "n_points": p.n, "build_s": build_s[q], "group_build_s": t1 - t0, "solve_s": t2 - t1,
                     "device_bytes": p.info()["device_bytes"], "response_bytes": hosts[q].numel() * 8,
                     "group_size": len(reqs)}
                if keep_solution:
                    o["x"] = hosts[q].numpy().reshape(1, p.n)
                outs.append(o)
            return outs
        finally:
            for p in plans:
                if p is not None:
                    p.close()

    return run


class ServingEngine:
    def __init__(self, executor=None, max_inflight: int = 64, budget_bytes: int | None = None,
                 budget_frac: float = 0.8, restart: int = 30, tol: float = 1e-4, stream_factory=None,
                 workers: int | None = None, max_iter: int = 1000, group_executor=None, group_max: int = 8,
                 group_n_max: int = 200_000, group_wait_s: float = 0.05):
        if budget_bytes is None:
            import torch

            budget_bytes = int(budget_frac * torch.cuda.mem_get_info()[1])
        self.admission = Admission(budget_bytes)
        self.max_inflight = int(workers if workers is not None else max_inflight)  # slots
        self.restart = int(restart)
        self.executor = executor if executor is not None else gpu_executor(restart, tol, max_iter=max_iter)
        # single right-hand-side requests of at most group_n_max points that arrive within
        # group_wait_s of each other are solved together (up to group_max): one shared launch per
        # restart cycle for all of them; group_max = 1 turns grouping off
        if group_executor is None and executor is None and group_max > 1:
            group_executor = gpu_group_executor(restart, tol, max_iter=max_iter)
        self.group_executor = group_executor
        self.group_max = int(group_max)
        self.group_n_max = int(group_n_max)
        self.group_wait_s = float(group_wait_s)
        if stream_factory is None:
            def stream_factory():
                import torch

                return torch.cuda.Stream()
        self.stream_factory = stream_factory

    def run(self, requests):
        """requests: dicts with arrival_s, V, F, k, nrhs, dirs (and anything else, passed
        through). Blocks until all are served; returns (records, summary)."""
        reqs = sorted(requests, key=lambda r: r["arrival_s"])
        records = []
        rec_lock = threading.Lock()
        slots = threading.Semaphore(self.max_inflight)
        t0 = time.perf_counter()
        running = []

        def serve(r, t_arrive, est, stream):
            rec = {"id": r.get("id"), "arrival_s": t_arrive - t0, "nrhs": r["nrhs"], "estimate_bytes": est}
            t_start = time.perf_counter()
            try:
                out = self.executor(r, stream)
                rec.update(out)
                rec["status"] = "ok" if out.get("status", 0) == 0 else "not converged"
            except Exception as e:  # the request fails; the server goes on
                rec.update(status="error", error=str(e))
            finally:
                self.admission.release(est)
                slots.release()
            t_done = time.perf_counter()
            rec.update(start_s=t_start - t0, done_s=t_done - t0, wait_s=t_start - t_arrive, latency_s=t_done - t_arrive)
            with rec_lock:
                records.append(rec)

        class Group:  # single right-hand-side requests collected for one group solve
            def __init__(self):
                self.members = []  # (request, arrival time, estimate)
                self.open = True
                self.full = threading.Event()

        group_lock = threading.Lock()
        current = [None]

        def serve_group(g, stream):
            g.full.wait(self.group_wait_s)  # the collection window (or until the group is full)
            with group_lock:
                g.open = False
            t_start = time.perf_counter()
            reqs_g = [m[0] for m in g.members]
            try:
                outs = self.group_executor(reqs_g, stream)
                err = None
            except Exception as e:  # the group fails; the server goes on
                outs, err = [{} for _ in reqs_g], str(e)
            finally:
                for m in g.members:
                    self.admission.release(m[2])
                    slots.release()
            t_done = time.perf_counter()
            for (r, t_arrive, est), out in zip(g.members, outs):
                rec = {"id": r.get("id"), "arrival_s": t_arrive - t0, "nrhs": r["nrhs"], "estimate_bytes": est}
                rec.update(out)
                if err is not None:
                    rec.update(status="error", error=err)
                else:
                    rec["status"] = "ok" if out.get("status", 0) == 0 else "not converged"
                rec.update(start_s=t_start - t0, done_s=t_done - t0, wait_s=t_start - t_arrive,
                           latency_s=t_done - t_arrive)
                with rec_lock:
                    records.append(rec)

        # the dispatcher: requests in arrival order; each starts as soon as a slot and its
        # memory are free (admission in order, so a large request is not overtaken)
        for r in reqs:
            delay = t0 + r["arrival_s"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            t_arrive = t0 + r["arrival_s"]  # the request exists from its arrival, even while the dispatcher waits
            V = np.asarray(r["V"], dtype=np.float64)
            extent = float((V.max(axis=0) - V.min(axis=0)).max()) if V.size else 0.0
            est = estimate_bytes(len(r["F"]) * 3, r["nrhs"], self.restart, float(r["k"]), extent)
            ticket = self.admission.ticket()
            slots.acquire()
            if not self.admission.acquire(ticket, est):
                slots.release()
                with rec_lock:
                    records.append({"id": r.get("id"), "arrival_s": t_arrive - t0, "nrhs": r["nrhs"],
                                    "estimate_bytes": est, "status": "rejected",
                                    "done_s": time.perf_counter() - t0})
                continue
            if (self.group_executor is not None and self.group_max > 1 and r["nrhs"] == 1 and
                    len(r["F"]) * 3 <= self.group_n_max):
                with group_lock:
                    g = current[0]
                    fresh = g is None or not g.open or len(g.members) >= self.group_max
                    if fresh:
                        g = current[0] = Group()
                    g.members.append((r, t_arrive, est))
                    if len(g.members) >= self.group_max:
                        g.full.set()
                if not fresh:
                    continue
                th = threading.Thread(target=serve_group, args=(g, self.stream_factory()))
            else:
                th = threading.Thread(target=serve, args=(r, t_arrive, est, self.stream_factory()))
            th.start()
            running.append(th)
        for th in running:
            th.join()
        return records, summarize(records, self.admission)


def summarize(records, admission=None):
    served = [r for r in records if r["status"] in ("ok", "not converged")]
    lat = np.array([r["latency_s"] for r in served]) if served else np.zeros(0)
    first = min((r["arrival_s"] for r in records), default=0.0)
    last = max((r["done_s"] for r in records), default=0.0)
    span = max(last - first, 1e-9)
    solved = sum(r["nrhs"] for r in records if r["status"] == "ok")
    out = {
        "requests": len(records), "ok": sum(r["status"] == "ok" for r in records),
        "not_converged": sum(r["status"] == "not converged" for r in records),
        "rejected": sum(r["status"] == "rejected" for r in records),
        "errors": sum(r["status"] == "error" for r in records),
        "solves": solved, "makespan_s": span, "solves_per_s": solved / span,
        "requests_per_s": len(served) / span,
        "latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "latency_mean_s": float(lat.mean()) if lat.size else None,
        "wait_mean_s": float(np.mean([r["wait_s"] for r in served])) if served else None,
        "build_mean_s": float(np.mean([r["build_s"] for r in served if "build_s" in r])) if served else None,
        "solve_mean_s": float(np.mean([r["solve_s"] for r in served if "solve_s" in r])) if served else None,
    }
    if admission is not None:
        out["budget_bytes"] = admission.budget
        out["peak_reserved_bytes"] = admission.peak
    return out
