"""Mixed-precision iterative refinement: GMRES on the fast plan (FP32 near field,
BF16x3 tensor-core M2L, p = 7, tolerance 1e-4) inside an outer loop whose
residuals r = b - A x use an accurate plan and are formed in double-float.  The
accurate plan (precision = 1, p = 14, FP32 SIMT M2L) evaluates its near field and
correction in FP64 on the double-float iterate; its far field is FP32.

The accurate operator's parts against the FP64 oracle (same tree, same order):
  near field (P2P over the near leaves)     1e-11   (FP64 arithmetic)
  correction (FP64 quadrature nodes)        1e-9
  far field (FP32 translations)             1e-6
Checked with the oracle's exact dense operator Z:
  refined to 5e-7:   |Z x - b| / |b| <= 1.1e-6,  |x - x_LU| / |x_LU| < 5e-4 (cond(Z) ~ 60)
  plain GMRES 1e-4:  the refined solution's residual is at least 20 times smaller
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _df(plan, s, parts):
    o = torch.empty(plan.n, 4, dtype=torch.float32, device="cuda")
    plan.matvec_df(pkg.df_from_complex(s), o, parts)
    torch.cuda.synchronize()
    return pkg.df_to_complex(o)


def test_accurate_operator_parts_against_oracle():
    V, F = synthetic.sphere_mesh(3)
    k, p = 1.0, 14
    plan = pkg.Plan(V, F, k, p_fixed=p, m2l_tensor=0, precision=1)
    try:
        X, W, _ = oracle.points(V, F)
        r = oracle.near_radius(V, F, 1.0)
        s = synthetic.random_density(plan.n, seed=11).astype(np.complex128)
        Zs = oracle.direct_matvec(V, F, k, r, s)
        nz = np.linalg.norm(Zs)
        near, info = oracle.fmm(X, W, k, s, leaf_max=64, p_fixed=p, parts=1)
        far, _ = oracle.fmm(X, W, k, s, leaf_max=64, p_fixed=p, parts=2)
        assert info[0] == plan.info()["depth"]
        corr = oracle.correction_csr(V, F, k, r) @ s
        assert np.linalg.norm(_df(plan, s, 1) - near) < 1e-11 * nz
        assert np.linalg.norm(_df(plan, s, 4) - corr) < 1e-9 * nz
        assert np.linalg.norm(_df(plan, s, 2) - far) < 1e-6 * nz
        assert np.linalg.norm(_df(plan, s, 7) - Zs) < 1e-6 * nz
        assert plan.device_status() == pkg.HFMM_OK
    finally:
        plan.close()


def test_matvec_df_needs_an_accurate_plan():
    V, F = synthetic.sphere_mesh(2)
    plan = pkg.Plan(V, F, 1.0, p_fixed=5)
    try:
        d = torch.zeros(plan.n, 4, dtype=torch.float32, device="cuda")
        with pytest.raises(pkg.HfmmError):
            plan.matvec_df(d, torch.empty_like(d))
    finally:
        plan.close()


def test_order_beyond_fp32_range_is_refused():
    """p = 18 on the N = 3,840 sphere at k = 1: the outgoing functions of the small boxes
    exceed FP32's range, so the plan is refused instead of returning NaN."""
    V, F = synthetic.sphere_mesh(3)
    with pytest.raises(pkg.HfmmError):
        pkg.Plan(V, F, 1.0, p_fixed=18, m2l_tensor=0)


def test_refinement_reaches_1e6_against_dense_operator():
    V, F = synthetic.sphere_mesh(3)
    inner = pkg.Plan(V, F, 1.0, p_fixed=7, m2l_tensor=1, restart=30, tol=1e-4)
    outer = pkg.Plan(V, F, 1.0, p_fixed=14, m2l_tensor=0, precision=1)
    try:
        b = torch.empty(inner.n, dtype=torch.complex64, device="cuda")
        inner.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, nout, nin, rr = inner.solve_refined(outer, b, x, tol=5e-7, max_outer=8)
        assert st == pkg.HFMM_OK and rr <= 5e-7 and 2 <= nout <= 8 and nin > 0
        xp = torch.empty_like(b)
        sp, _, rp = inner.solve(b, xp)
        assert sp == pkg.HFMM_OK and rp[0] <= 1e-4
        X, _, _ = oracle.points(V, F)
        Z = oracle.dense_Z(V, F, 1.0, oracle.near_radius(V, F, 1.0))
        bb = b.cpu().numpy().astype(np.complex128)
        xr = x.cpu().numpy().astype(np.complex128)
        xpl = xp.cpu().numpy().astype(np.complex128)
        res_ref = np.linalg.norm(Z @ xr - bb) / np.linalg.norm(bb)
        res_plain = np.linalg.norm(Z @ xpl - bb) / np.linalg.norm(bb)
        assert res_ref <= 1.1e-6
        assert res_ref * 20 < res_plain
        assert _rel(xr, np.linalg.solve(Z, bb)) < 5e-4
    finally:
        inner.close()
        outer.close()


def test_refinement_rejects_plans_of_different_meshes():
    V2, F2 = synthetic.sphere_mesh(2)
    V3, F3 = synthetic.sphere_mesh(3)
    a = pkg.Plan(V2, F2, 1.0, p_fixed=5)
    c = pkg.Plan(V3, F3, 1.0, p_fixed=5)
    try:
        b = torch.zeros(a.n, dtype=torch.complex64, device="cuda")
        with pytest.raises(pkg.HfmmError):
            pkg.hfmm_solve_refined(a.handle, c.handle, b, torch.empty_like(b))
    finally:
        a.close()
        c.close()
