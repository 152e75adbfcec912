"""Mixed-precision iterative refinement: GMRES on the fast plan (FP32 near field,
BF16x3 tensor-core M2L, p = 7, tolerance 1e-4) inside an outer loop whose
residuals r = b - A x use an accurate plan (p = 14, FP32 SIMT M2L) and are formed
in double-float. Checked with the oracle's exact dense operator Z:
  refined to 1e-6:   |Z x - b| / |b| < 3e-6,  |x - x_LU| / |x_LU| < 5e-4 (cond(Z) ~ 60)
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


def test_refinement_reaches_1e6_against_dense_operator():
    V, F = synthetic.sphere_mesh(3)
    inner = pkg.Plan(V, F, 1.0, p_fixed=7, m2l_tensor=1, restart=30, tol=1e-4)
    outer = pkg.Plan(V, F, 1.0, p_fixed=14, m2l_tensor=0)
    try:
        b = torch.empty(inner.n, dtype=torch.complex64, device="cuda")
        inner.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, nout, nin, rr = inner.solve_refined(outer, b, x, tol=1e-6, max_outer=8)
        assert st == pkg.HFMM_OK and rr <= 1e-6 and 2 <= nout <= 8 and nin > 0
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
        assert res_ref < 3e-6
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
