"""The scratch-free point sum, checked against the plan-based entry point.

hfmm_point_sum_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool or arena, processes whose device
footprint must stay fixed); it keeps its working set in a fixed device array.
Its output must match hfmm_matvec_parts(parts = 1) on a plan whose single leaf
holds every point, within the near-field tolerance of the other GPU tests
(1e-5 relative 2-norm), on consecutive calls that reuse the array.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_plan_near_field_on_consecutive_calls():
    V, F = synthetic.sphere_mesh(2)
    k = 3.0
    plan = pkg.Plan(V, F, k, leaf_max=10 ** 6)
    try:
        assert plan.info()["depth"] == 0  # one leaf: the near field is every pair
        X, W, _ = plan.points()
        xyz = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        w = torch.from_numpy(np.ascontiguousarray(W)).cuda()
        for seed in (11, 12):
            s = synthetic.random_density(plan.n, seed=seed)
            d = torch.from_numpy(s.astype(np.complex64)).cuda()
            ref = torch.empty_like(d)
            plan.matvec_parts(d, ref, 1)
            out = torch.full_like(d, complex(np.nan, np.nan))
            assert pkg.hfmm_point_sum_noalloc(xyz, w, d, out, k) == pkg.HFMM_OK
            torch.cuda.synchronize()
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert _rel(got.astype(np.complex128), want.astype(np.complex128)) < 1e-5
    finally:
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_capacity():
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.complex64, device="cuda")
    n = pkg.HFMM_NOALLOC_MAX_POINTS + 1
    st = pkg.lib().hfmm_point_sum_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()), n, 1.0,
                                          ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), None)
    assert st == pkg.HFMM_E_OVERFLOW
    assert "exceeds the scratch capacity" in pkg.hfmm_last_error()
