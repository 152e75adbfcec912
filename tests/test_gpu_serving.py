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
    eng = serving.ServingEngine(workers=2, restart=30, tol=1e-4)
    recs, summ = eng.run(reqs)
    assert summ["ok"] == len(specs) and summ["solves"] == sum(s[3] for s in specs)
    for r in recs:
        assert r["status"] == "ok"
        assert len(r["relres"]) == r["nrhs"] and max(r["relres"]) <= 1e-4
        assert r["latency_s"] >= r["build_s"] + r["solve_s"] - 1e-3
    assert summ["latency_p99_s"] >= summ["latency_p50_s"] > 0


def test_results_alone_equal_results_in_the_mix():
    """Two workers serve four overlapping requests (plans built while others solve); each
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
    mix, summ = serving.ServingEngine(executor=ex, workers=2, restart=30).run(reqs)
    assert summ["ok"] == len(specs), [(r["id"], r["status"], r.get("relres")) for r in mix]
    got = {r["id"]: r for r in mix}
    for r in reqs:
        alone, s1 = serving.ServingEngine(executor=ex, workers=1, restart=30).run([dict(r)])
        assert s1["ok"] == 1
        xa, xm = alone[0]["x"].astype(np.complex128), got[r["id"]]["x"].astype(np.complex128)
        assert xa.shape == xm.shape == (r["nrhs"], 3 * len(r["F"]))
        for q in range(r["nrhs"]):
            assert np.linalg.norm(xm[q] - xa[q]) <= 2e-3 * np.linalg.norm(xa[q]), (r["id"], q)
