"""Serving loop, host logic: admission by a memory budget in arrival order,
rejection of requests that can never fit, latency accounting, and the request
generator's distributions. The executor is a stand-in that sleeps (no GPU)."""
import threading
import time

import numpy as np

import synthetic
from paper_1803_09948_gb300 import serving


def _fake_executor(log, lock, dt=0.05):
    def run(req, stream):
        with lock:
            log.append(("start", req["id"], time.perf_counter()))
        time.sleep(dt)
        with lock:
            log.append(("end", req["id"], time.perf_counter()))
        return {"status": 0, "iterations": [1] * req["nrhs"], "relres": [1e-5] * req["nrhs"], "build_s": 0.0,
                "solve_s": dt}
    return run


def _req(i, t, n_tri, nrhs=1):
    return {"id": i, "arrival_s": t, "V": np.zeros((3, 3)), "F": np.zeros((n_tri, 3), dtype=np.int32), "k": 1.0,
            "nrhs": nrhs, "dirs": [[0.0, 0.0, 1.0]] * nrhs}


def test_budget_limits_concurrency_and_keeps_arrival_order():
    log, lock = [], threading.Lock()
    one = serving.estimate_bytes(3 * 1000, 1, 30)
    eng = serving.ServingEngine(executor=_fake_executor(log, lock), max_inflight=4, budget_bytes=2 * one + 1,
                                restart=30, stream_factory=lambda: None)
    reqs = [_req(i, 0.001 * i, 1000) for i in range(8)]
    recs, summ = eng.run(reqs)
    assert summ["ok"] == 8 and summ["rejected"] == 0
    # never more than two in flight: the budget holds two estimates
    live, peak = 0, 0
    for kind, _, _ in sorted(log, key=lambda e: e[2]):
        live += 1 if kind == "start" else -1
        peak = max(peak, live)
    assert peak <= 2 and summ["peak_reserved_bytes"] <= 2 * one + 1
    starts = [i for kind, i, _ in sorted(log, key=lambda e: e[2]) if kind == "start"]
    assert starts == sorted(starts)  # admitted in arrival order
    for r in recs:
        assert r["latency_s"] >= r["solve_s"] - 1e-3 and r["wait_s"] >= 0


def test_memory_not_a_worker_count_bounds_concurrency():
    """64 slots, a budget of six requests: six run at once, then each finished request lets the
    next one in (admission follows memory, not a fixed pool of workers)."""
    log, lock = [], threading.Lock()
    one = serving.estimate_bytes(3 * 1000, 1, 30)
    eng = serving.ServingEngine(executor=_fake_executor(log, lock, 0.1), max_inflight=64, budget_bytes=6 * one,
                                restart=30, stream_factory=lambda: None)
    recs, summ = eng.run([_req(i, 0.0, 1000) for i in range(12)])
    live, peak = 0, 0
    for kind, _, _ in sorted(log, key=lambda e: e[2]):
        live += 1 if kind == "start" else -1
        peak = max(peak, live)
    assert summ["ok"] == 12 and peak == 6
    assert summ["makespan_s"] < 0.35  # two waves of 0.1 s, not twelve


def test_single_rhs_requests_are_grouped():
    """Small single right-hand-side requests arriving together are served as groups of at most
    group_max (one group solve each); a multi-RHS request runs on its own; every request keeps
    its own record, and its latency includes the collection window."""
    log, lock = [], threading.Lock()
    groups = []

    def group_exec(reqs, stream):
        with lock:
            groups.append([r["id"] for r in reqs])
        time.sleep(0.05)
        return [{"status": 0, "iterations": [3], "relres": [1e-5], "build_s": 0.0, "solve_s": 0.05,
                 "group_size": len(reqs)} for _ in reqs]

    eng = serving.ServingEngine(executor=_fake_executor(log, lock, 0.05), group_executor=group_exec, group_max=4,
                                group_wait_s=0.05, budget_bytes=10 ** 12, restart=30, stream_factory=lambda: None)
    reqs = [_req(i, 0.002 * i, 1000) for i in range(6)] + [_req(6, 0.003, 1000, nrhs=3)]
    recs, summ = eng.run(reqs)
    assert summ["ok"] == 7
    assert sorted(len(g) for g in groups) == [2, 4] and sorted(sum(groups, [])) == list(range(6))
    by = {r["id"]: r for r in recs}
    assert [e[1] for e in log if e[0] == "start"] == [6]  # the multi-RHS request alone
    for i in range(6):
        assert by[i]["group_size"] in (2, 4) and by[i]["latency_s"] >= 0.05


def test_oversized_request_is_rejected_and_others_served():
    log, lock = [], threading.Lock()
    eng = serving.ServingEngine(executor=_fake_executor(log, lock, 0.01), max_inflight=2,
                                budget_bytes=serving.estimate_bytes(3 * 2000, 1, 30), restart=30,
                                stream_factory=lambda: None)
    reqs = [_req(0, 0.0, 1000), _req(1, 0.001, 10 ** 6, nrhs=16), _req(2, 0.002, 1000)]
    recs, summ = eng.run(reqs)
    st = {r["id"]: r["status"] for r in recs}
    assert st == {0: "ok", 1: "rejected", 2: "ok"} and summ["solves"] == 2


def test_latency_includes_waiting_for_the_budget():
    log, lock = [], threading.Lock()
    one = serving.estimate_bytes(3 * 1000, 1, 30)
    eng = serving.ServingEngine(executor=_fake_executor(log, lock, 0.1), max_inflight=2, budget_bytes=one,
                                restart=30, stream_factory=lambda: None)
    recs, summ = eng.run([_req(0, 0.0, 1000), _req(1, 0.0, 1000)])
    second = max(recs, key=lambda r: r["done_s"])
    assert second["wait_s"] > 0.08 and second["latency_s"] > 0.18
    assert summ["latency_p99_s"] >= summ["latency_p50_s"] > 0.09


def test_request_generator_distributions():
    reqs = synthetic.serving_requests(2000, seed=1, rate=20.0)
    gaps = np.diff([0.0] + [r["arrival_s"] for r in reqs])
    assert abs(np.mean(gaps) - 0.05) < 0.005  # Poisson arrivals, mean 20 per second
    n = np.array([r["n_points"] for r in reqs])
    assert n.min() >= 0.9 * 10_000 and n.max() <= 1.1 * 1_000_000
    assert np.all(n % 60 == 0)  # N = 60 nu^2
    ln = np.log(n)
    assert abs(np.median(ln) - 0.5 * (np.log(1e4) + np.log(1e6))) < 0.2  # log-uniform
    assert {r["shape"] for r in reqs} == {"sphere", "ellipsoid", "star"}
    assert min(r["nrhs"] for r in reqs) == 1 and max(r["nrhs"] for r in reqs) == 16
    k = np.array([r["k"] for r in reqs])
    assert 1.0 <= k.min() and k.max() <= 30.0


def test_geodesic_meshes_are_closed_and_outward():
    for nu in (1, 3, 7):
        v, f = synthetic.geodesic_sphere(nu)
        assert f.shape[0] == 20 * nu * nu and v.shape[0] == 10 * nu * nu + 2
        e = np.sort(np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]]), axis=1)
        _, cnt = np.unique(e, axis=0, return_counts=True)
        assert np.all(cnt == 2)
        nrm = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
        assert np.all((nrm * v[f].mean(1)).sum(1) > 0)
    v, f = synthetic.serving_shape("ellipsoid", 4, seed=0)
    assert np.isclose(np.abs(v[:, 0]).max(), 2.0)
    v, f = synthetic.serving_shape("star", 4, seed=3)
    r = np.linalg.norm(v, axis=1)
    assert 0.8 - 1e-12 <= r.min() and r.max() <= 1.2 + 1e-12
