"""Plan building: the projection of the translation operators (M2L, M2M, L2L) runs its
quadrature sums in double-float arithmetic on the FP32 pipes.  Checked against the same
projection in FP64 (HFMM_PROJECTION_FP64=1 forces that kernel) on a k = 30 plan whose coarse
levels take orders 21 and 13: the two FP32-stored operator sets may differ in the last bit,
so the far fields agree to 1e-6; and the matvec against the oracle's FP64 direct sum."""
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


def _apply(plan, s, parts):
    d = torch.from_numpy(s.astype(np.complex64)).cuda()
    o = torch.empty_like(d)
    plan.matvec_parts(d, o, parts)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128)


def test_double_float_projection_matches_fp64(monkeypatch):
    V, F = synthetic.serving_shape("star", 13, 3)
    k = 30.0
    monkeypatch.setenv("HFMM_PROJECTION_FP64", "1")
    ref = pkg.Plan(V, F, k, m2l_tensor=0)
    monkeypatch.delenv("HFMM_PROJECTION_FP64")
    fast = pkg.Plan(V, F, k, m2l_tensor=0)
    try:
        assert fast.info()["orders"][2] >= 20
        s = synthetic.random_density(fast.n, seed=2)
        far_ref, far = _apply(ref, s, 2), _apply(fast, s, 2)
        assert np.linalg.norm(far - far_ref) <= 1e-6 * np.linalg.norm(far_ref)
        rows = np.random.default_rng(0).choice(fast.n, 300, replace=False)
        exact = oracle.direct_rows(V, F, k, oracle.near_radius(V, F, 1.0), rows, s)
        got = _apply(fast, s, 7)[rows]
        assert np.linalg.norm(got - exact) <= 1e-4 * np.linalg.norm(exact)
    finally:
        ref.close()
        fast.close()
