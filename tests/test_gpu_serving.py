"""Serving loop on the GPU: a few small requests of each shape (geodesic meshes,
several wavenumbers, 1 to 4 right-hand sides) through the real executor; every
right-hand side converges to the tolerance and the records add up."""
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
