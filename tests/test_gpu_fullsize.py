"""Full-size parity: the benchmark's sphere workloads in the benchmark's own
configuration (default per-level orders, tensor-core translations at the levels
with (p+1)^2 <= 64, FP32 SIMT above), checked on sampled rows against the
oracle's FP64 direct summation of the discretised operator (point part plus the
exact self/near integrals).

Tolerances (relative 2-norm over the sampled rows):
  FMM matvec vs direct summation        1e-4  (the matvec bar)
  tensor-core vs FP32 SIMT far field    3e-5  (BF16 split in three products)
The sample always contains the first and the last point (ends of the Morton order
and of the last, ragged leaf) besides seeded random rows.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu

WORKLOADS = [("sphere_163840", 10.0), ("sphere_655360", 20.0)]
SAMPLE = 256


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    r = rng.choice(n, size=min(SAMPLE, n), replace=False)
    return np.unique(np.concatenate([r, [0, n - 1]]))


def _matvec(plan, s, parts=7):
    d = torch.from_numpy(s.astype(np.complex64)).cuda()
    o = torch.empty_like(d)
    if parts == 7:
        plan.matvec(d, o)
    else:
        plan.matvec_parts(d, o, parts)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,k", WORKLOADS)
def test_fullsize_matvec_sampled_rows_against_direct_sum(name, k):
    V, F = synthetic.workload_mesh(name)
    plan = pkg.Plan(V, F, k)
    try:
        assert plan.n == 3 * F.shape[0]
        orders = plan.info()["orders"][2:]
        # both translation paths are exercised: a level above the tensor-core order limit
        # ((p+1)^2 > 64, FP32 SIMT) and levels on the tensor cores
        assert max(orders) > 7 and min(orders) <= 7
        s = synthetic.random_density(plan.n, seed=3)
        got = _matvec(plan, s)
        assert plan.device_status() == pkg.HFMM_OK
        assert np.all(np.isfinite(got))
        rows = _rows(plan.n, seed=5)
        ref = oracle.direct_rows(V, F, k, oracle.near_radius(V, F, plan.cfg.near_factor), rows, s)
        assert _rel(got[rows], ref) < 1e-4
    finally:
        plan.close()


def test_fullsize_solve_true_residual_against_oracle():
    """GMRES(50) to 1e-4 on the 1.97 M-point sphere at k = 20 (the single large solve):
    the solution's true residual b - Z x, with Z the oracle's exact FP64 operator, on
    1,024 sampled rows (plus the two ends), is within 1e-4 + 10 %."""
    name, k = WORKLOADS[1]
    V, F = synthetic.workload_mesh(name)
    plan = pkg.Plan(V, F, k, restart=50, tol=1e-4)
    try:
        b = torch.empty(plan.n, dtype=torch.complex64, device="cuda")
        plan.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, its, rr = plan.solve(b, x)
        assert st == pkg.HFMM_OK and rr[0] <= 1e-4
        torch.cuda.synchronize()
        xg = x.cpu().numpy().astype(np.complex128)
        rng = np.random.default_rng(21)
        rows = np.unique(np.concatenate([rng.choice(plan.n, 1024, replace=False), [0, plan.n - 1]]))
        X, _, _ = oracle.points(V, F)
        zx = oracle.direct_rows(V, F, k, oracle.near_radius(V, F, plan.cfg.near_factor), rows, xg)
        bb = oracle.plane_wave(X[rows], k, (0.0, 0.0, 1.0))
        assert np.linalg.norm(zx - bb) / np.linalg.norm(bb) <= 1.1e-4
    finally:
        plan.close()


def test_fullsize_tensor_core_far_field_against_simt():
    name, k = WORKLOADS[0]
    V, F = synthetic.workload_mesh(name)
    tc = pkg.Plan(V, F, k, m2l_tensor=1)
    simt = pkg.Plan(V, F, k, m2l_tensor=0)
    try:
        s = synthetic.random_density(tc.n, seed=4)
        far_tc = _matvec(tc, s, parts=2)
        far_simt = _matvec(simt, s, parts=2)
        assert tc.device_status() == pkg.HFMM_OK
        assert _rel(far_tc, far_simt) < 3e-5
    finally:
        tc.close()
        simt.close()
