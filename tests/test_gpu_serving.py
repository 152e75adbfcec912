"""Serving loop on the GPU: a few small requests of each shape (geodesic meshes,
several wavenumbers, 1 to 4 right-hand sides) through the real executor; every
right-hand side converges to the tolerance and the records add up, and each
request's solutions served in the mix equal those of the same request served alone."""
import numpy as np
import pytest

import synthetic
from paper_1803_09948_gb300 import serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def test_small_requests_are_served():
    specs = [("sphere", 8, 2.0, 1), ("ellipsoid", 9, 3.0, 3), ("star", 10, 1.5, 4), ("sphere", 12, 4.0, 2)]
    reqs = []
    for q, (shape, nu, k, nrhs) in enumerate(specs):
        V, F = synthetic.serving_shape(shape, nu, seed=q)
        dirs = np.asarray(synthetic.fibonacci_directions(nrhs, seed=q)).reshape(nrhs, 3)
        reqs.append({"id": q, "arrival_s": 0.02 * q, "V": V, "F": F, "k": k, "nrhs": nrhs, "dirs": dirs})
    eng = serving.ServingEngine(restart=30, tol=1e-4)
    recs, summ = eng.run(reqs)
    assert summ["ok"] == len(specs) and summ["solves"] == sum(s[3] for s in specs)
    for r in recs:
        assert r["status"] == "ok"
        assert len(r["relres"]) == r["nrhs"] and max(r["relres"]) <= 1e-4
        assert r["latency_s"] >= r["build_s"] + r["solve_s"] - 1e-3
    assert summ["latency_p99_s"] >= summ["latency_p50_s"] > 0


def test_results_alone_equal_results_in_the_mix():
    """Four overlapping requests served at once (plans built while others solve); each
    request is then served alone.  GMRES runs to 1e-5 on both sides (the FP32 operator's
    reduction-order noise floors some of these residuals near 1e-6), so two solutions of
    one request may differ by up to 2 cond(Z) x 1e-5 = 2e-3 (cond(Z) <= 100 here); a
    request that read another's buffers or stream would differ at O(1)."""
    specs = [("sphere", 8, 2.0, 2), ("ellipsoid", 9, 3.0, 1), ("star", 8, 1.5, 3), ("sphere", 10, 4.0, 1)]
    reqs = []
    for q, (shape, nu, k, nrhs) in enumerate(specs):
        V, F = synthetic.serving_shape(shape, nu, seed=10 + q)
        dirs = np.asarray(synthetic.fibonacci_directions(nrhs, seed=q)).reshape(nrhs, 3)
        reqs.append({"id": q, "arrival_s": 0.0, "V": V, "F": F, "k": k, "nrhs": nrhs, "dirs": dirs})
    ex = serving.gpu_executor(restart=30, tol=1e-5, keep_solution=True)
    mix, summ = serving.ServingEngine(executor=ex, restart=30).run(reqs)
    assert summ["ok"] == len(specs), [(r["id"], r["status"], r.get("relres")) for r in mix]
    got = {r["id"]: r for r in mix}
    for r in reqs:
        alone, s1 = serving.ServingEngine(executor=ex, max_inflight=1, restart=30).run([dict(r)])
        assert s1["ok"] == 1
        xa, xm = alone[0]["x"].astype(np.complex128), got[r["id"]]["x"].astype(np.complex128)
        assert xa.shape == xm.shape == (r["nrhs"], 3 * len(r["F"]))
        for q in range(r["nrhs"]):
            assert np.linalg.norm(xm[q] - xa[q]) <= 2e-3 * np.linalg.norm(xa[q]), (r["id"], q)


def test_served_solutions_match_the_oracle():
    """Small requests (N = 60 nu^2 = 1,500 .. 2,160 points) served together; every right-hand
    side's solution against the oracle's exact dense operator Z: the residual |Z x - b| / |b|
    is the FMM operator's error (p from the per-level formula, <= 1e-4) plus the GMRES
    tolerance (1e-5), and x is within cond(Z) times that of the LU solution (cond(Z) < 100
    for these shapes and wavenumbers)."""
    import oracle

    specs = [("sphere", 6, 2.0, 2), ("ellipsoid", 5, 3.0, 1), ("star", 6, 1.5, 2)]
    reqs = []
    for q, (shape, nu, k, nrhs) in enumerate(specs):
        V, F = synthetic.serving_shape(shape, nu, seed=20 + q)
        dirs = np.asarray(synthetic.fibonacci_directions(nrhs, seed=q)).reshape(nrhs, 3)
        reqs.append({"id": q, "arrival_s": 0.01 * q, "V": V, "F": F, "k": k, "nrhs": nrhs, "dirs": dirs})
    ex = serving.gpu_executor(restart=30, tol=1e-5, keep_solution=True)
    recs, summ = serving.ServingEngine(executor=ex, restart=30).run(reqs)
    assert summ["ok"] == len(specs)
    got = {r["id"]: r for r in recs}
    for r in reqs:
        V, F, k = r["V"], r["F"], r["k"]
        X, _, _ = oracle.points(V, F)
        Z = oracle.dense_Z(V, F, k, oracle.near_radius(V, F, 1.0))
        for q in range(r["nrhs"]):
            b = oracle.plane_wave(X, k, r["dirs"][q])
            x = got[r["id"]]["x"][q].astype(np.complex128)
            assert np.linalg.norm(Z @ x - b) <= 2e-4 * np.linalg.norm(b), (r["id"], q)
            x_lu = np.linalg.solve(Z, b)
            assert np.linalg.norm(x - x_lu) <= 2e-2 * np.linalg.norm(x_lu), (r["id"], q)


def test_grouped_requests_equal_requests_alone():
    """Single right-hand-side requests arriving together are served as one group solve (every
    restart cycle of all of them in one graph launch); each one's solution equals the same
    request served alone, within 2 cond(Z) x 1e-5 (cond(Z) <= 100 here)."""
    specs = [("sphere", 8, 2.0), ("ellipsoid", 7, 3.0), ("star", 8, 1.5), ("sphere", 6, 1.0)]
    reqs = []
    for q, (shape, nu, k) in enumerate(specs):
        V, F = synthetic.serving_shape(shape, nu, seed=50 + q)
        dirs = np.asarray(synthetic.fibonacci_directions(1, seed=q)).reshape(1, 3)
        reqs.append({"id": q, "arrival_s": 0.001 * q, "V": V, "F": F, "k": k, "nrhs": 1, "dirs": dirs})
    ex = serving.gpu_executor(restart=30, tol=1e-5, keep_solution=True)
    gx = serving.gpu_group_executor(restart=30, tol=1e-5, keep_solution=True)
    recs, summ = serving.ServingEngine(executor=ex, group_executor=gx, group_max=8, group_wait_s=0.2,
                                       restart=30).run(reqs)
    assert summ["ok"] == len(specs)
    got = {r["id"]: r for r in recs}
    assert all(got[r["id"]]["group_size"] == len(specs) for r in reqs)
    for r in reqs:
        alone, s1 = serving.ServingEngine(executor=ex, max_inflight=1, group_max=1, restart=30).run([dict(r)])
        assert s1["ok"] == 1
        xa, xg = alone[0]["x"].astype(np.complex128), got[r["id"]]["x"].astype(np.complex128)
        assert np.linalg.norm(xg[0] - xa[0]) <= 2e-3 * np.linalg.norm(xa[0]), r["id"]
