"""The scratch-free point sum (hfmm_point_sum_noalloc).

It serves callers that cannot allocate device memory: code running inside
another framework's memory pool or arena, where cudaMalloc is not theirs to
call, and processes whose device footprint must stay fixed after start-up.
Its working set lives in one fixed device array that every call shares.

Checked here, within the near-field tolerance of the other GPU tests (1e-5
relative 2-norm):
  * against the plan-based entry point (hfmm_matvec_parts, parts = 1, on a plan
    whose single leaf holds every point) on two calls in a row;
  * against the FP64 oracle's point sum, all rows at N = 960 and sampled rows at
    N = 40,560 (k = 20) and N = 261,360 (k = 30, near the array's capacity), where
    |k x| is largest and close pairs are most exposed to rounding;
  * that repeated calls leave the device's free memory unchanged, and that bad
    arguments and sizes beyond the capacity are refused with a message.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _inputs(V, F, seed):
    X, W, _ = oracle.points(V, F)
    s = synthetic.random_density(X.shape[0], seed=seed)
    return X, W, s


def _noalloc(X, W, s, k, stream=None):
    xyz = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    w = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    d = torch.from_numpy(s.astype(np.complex64)).cuda()
    out = torch.full_like(d, complex(np.nan, np.nan))
    assert pkg.hfmm_point_sum_noalloc(xyz, w, d, out, k, stream=stream) == pkg.HFMM_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


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
            assert _rel(got.astype(np.complex128), want.astype(np.complex128)) < TOL
            # and both against the oracle's FP64 point sum
            assert _rel(got.astype(np.complex128), oracle.point_sum(X, W, k, s)) < TOL
    finally:
        plan.close()


@pytest.mark.parametrize("nu,k", [(26, 20.0), (66, 30.0)])
def test_noalloc_large_k_against_oracle_sampled_rows(nu, k):
    """Geodesic spheres of N = 60 nu^2 points (40,560 and 261,360 <= the capacity
    262,144) at the top of the configurations' wavenumbers: |k (x - x_0)| reaches 2k."""
    V, F = synthetic.geodesic_sphere(nu)
    X, W, s = _inputs(V, F, seed=nu)
    assert X.shape[0] <= pkg.HFMM_NOALLOC_MAX_POINTS
    got = _noalloc(X, W, s, k)
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(nu)
    rows = np.unique(np.concatenate([rng.choice(X.shape[0], 256, replace=False), [0, X.shape[0] - 1]]))
    ref = oracle.point_sum_rows(X, W, k, s, rows)
    assert _rel(got[rows], ref) < TOL


def test_noalloc_on_a_side_stream_and_ragged_sizes():
    """A caller's own stream; sizes that leave a partial block (n = 1, 257, 960)."""
    V, F = synthetic.sphere_mesh(2)
    X, W, s = _inputs(V, F, seed=4)
    st = torch.cuda.Stream()
    for n in (1, 257, X.shape[0]):
        with torch.cuda.stream(st):
            got = _noalloc(X[:n], W[:n], s[:n], 2.0, stream=st)
        ref = oracle.point_sum(X[:n], W[:n], 2.0, s[:n])
        if n == 1:
            assert got[0] == 0
        else:
            assert _rel(got, ref) < TOL


def test_noalloc_repeat_calls_leave_free_memory_unchanged():
    V, F = synthetic.sphere_mesh(3)
    X, W, s = _inputs(V, F, seed=6)
    xyz = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    w = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    d = torch.from_numpy(s.astype(np.complex64)).cuda()
    out = torch.empty_like(d)
    assert pkg.hfmm_point_sum_noalloc(xyz, w, d, out, 5.0) == pkg.HFMM_OK  # loads the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert pkg.hfmm_point_sum_noalloc(xyz, w, d, out, 5.0) == pkg.HFMM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def _raw(x, w, n, k, d, o):
    return pkg.lib().hfmm_point_sum_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()), n, k,
                                            ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(o.data_ptr()), None)


def test_noalloc_rejects_sizes_beyond_its_capacity_and_bad_arguments():
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.complex64, device="cuda")
    assert _raw(x, w, pkg.HFMM_NOALLOC_MAX_POINTS + 1, 1.0, d, d) == pkg.HFMM_E_OVERFLOW
    assert "exceeds the scratch capacity" in pkg.hfmm_last_error()
    for k in (float("inf"), float("nan"), 0.0, -1.0):
        assert _raw(x, w, 1, k, d, d) == pkg.HFMM_E_INVALID
        assert "k must be finite and positive" in pkg.hfmm_last_error()
    assert _raw(x, w, 0, 1.0, d, d) == pkg.HFMM_E_INVALID
    assert "n must be positive" in pkg.hfmm_last_error()
