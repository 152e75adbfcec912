"""Adaptive octree (config adaptive = 1) through the C ABI on a sphere whose cap carries 16
times the point density of the rest (leaves at two to three depths; the far field uses the
M2L, M2P and P2L lists):

  matvec vs the oracle's FP64 direct sum on sampled rows      1e-4  (p = 8 and 10: the fixed-
                                                                     order and any-order P2M/L2P)
  adaptive vs uniform plan, same orders                         1e-4
  near field alone vs the oracle's point sum over the leaves   1e-5  (FP32 P2P; the direct pairs
  touching each target's leaf (restated from the definition)          are exactly these)
  GMRES on the adaptive plan: converges to 1e-4, within 1e-3 of the uniform plan's solution
  three right-hand sides (run one at a time) equal three single matvecs     5e-6  (reduction order)
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


@pytest.fixture(scope="module")
def cap():
    V, F = synthetic.refined_cap_sphere(3, 4)  # 5,952 triangles, N = 17,856
    return V, F, 2.0


def _mv(plan, s, parts=7):
    d = torch.from_numpy(np.ascontiguousarray(s).astype(np.complex64)).cuda()
    o = torch.empty_like(d)
    if parts == 7:
        plan.matvec(d, o)
    else:
        plan.matvec_parts(d, o, parts)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("p", [8, 10])
def test_adaptive_matvec_against_oracle_rows(cap, p):
    V, F, k = cap
    plan = pkg.Plan(V, F, k, adaptive=1, leaf_max=32, p_fixed=p)
    try:
        info = plan.info()
        assert info["depth"] >= 4 and plan.device_status() == pkg.HFMM_OK
        s = synthetic.random_density(plan.n, seed=3)
        got = _mv(plan, s)
        rr = oracle.near_radius(V, F, plan.cfg.near_factor)
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([rng.choice(plan.n, 300, replace=False), [0, plan.n - 1]]))
        ref = oracle.direct_rows(V, F, k, rr, rows, s)
        assert _rel(got[rows], ref) < 1e-4
        uni = pkg.Plan(V, F, k, leaf_max=32, p_fixed=p)
        try:
            assert uni.info()["m2l_translations"] > 2 * info["m2l_translations"]
            assert _rel(got, _mv(uni, s)) < 1e-4
        finally:
            uni.close()
    finally:
        plan.close()


def _leaves(X, leaf_max):
    """Leaves of the adaptive tree from its definition (a box splits while it holds more than
    leaf_max points): each point's leaf, and each leaf's closed box in level-20 units."""
    mn, mx = X.min(0), X.max(0)
    ext = float(np.max(mx - mn))
    D = 1.0
    while D < ext:
        D *= 2.0
    while D * 0.5 >= ext:
        D *= 0.5
    lo = 0.5 * (mn + mx) - 0.5 * D
    q = np.clip(np.floor((X - lo) * (2.0 ** 20 / D)), 0, 2 ** 20 - 1).astype(np.int64)
    leaf_of = np.empty(X.shape[0], dtype=np.int64)
    blo, bhi = [], []
    stack = [(0, np.arange(X.shape[0]))]
    while stack:
        l, idx = stack.pop()
        if len(idx) <= leaf_max:
            leaf_of[idx] = len(blo)
            c = q[idx[0]] >> (20 - l)
            blo.append(c << (20 - l))
            bhi.append((c + 1) << (20 - l))
            continue
        ch = q[idx] >> (20 - (l + 1))
        keys, inv = np.unique(ch, axis=0, return_inverse=True)
        for j in range(len(keys)):
            stack.append((l + 1, idx[inv.ravel() == j]))
    return leaf_of, np.array(blo), np.array(bhi)


def test_adaptive_near_field_against_point_sum(cap):
    """parts = 1 (near field only): every target's sum over the points of the leaves that
    touch its leaf, against the oracle's point sum over exactly those sources (sampled)."""
    V, F, k = cap
    plan = pkg.Plan(V, F, k, adaptive=1, leaf_max=32, p_fixed=8)
    try:
        X, W, _ = plan.points()
        s = synthetic.random_density(plan.n, seed=7)
        got = _mv(plan, s, parts=1)
        leaf_of, blo, bhi = _leaves(X, 32)
        assert plan.info()["n_leaves"] == len(blo)
        rng = np.random.default_rng(11)
        for i in rng.choice(plan.n, 40, replace=False):
            t = leaf_of[i]
            touch = np.all((blo[t] <= bhi) & (blo <= bhi[t]), axis=1)
            src = np.flatnonzero(touch[leaf_of])
            sel = np.concatenate([[i], src[src != i]])
            ref = oracle.point_sum(X[sel], W[sel], k, s[sel])[0]  # target i against its direct sources
            assert abs(got[i] - ref) <= 1e-5 * max(abs(ref), 1e-3 * np.abs(got).max())
    finally:
        plan.close()


def test_adaptive_solve_and_several_rhs(cap):
    V, F, k = cap
    ad = pkg.Plan(V, F, k, adaptive=1, leaf_max=32, restart=50)
    uni = pkg.Plan(V, F, k, leaf_max=32, restart=50)
    try:
        b = torch.empty(ad.n, dtype=torch.complex64, device="cuda")
        ad.rhs_planewave([0.0, 0.6, 0.8], b)
        xa, xu = torch.empty_like(b), torch.empty_like(b)
        sa, ita, rra = ad.solve(b, xa)
        su, itu, rru = uni.solve(b, xu)
        assert sa == pkg.HFMM_OK and su == pkg.HFMM_OK and rra[0] <= 1e-4
        xa_h, xu_h = xa.cpu().numpy().astype(np.complex128), xu.cpu().numpy().astype(np.complex128)
        assert _rel(xa_h, xu_h) < 1e-3
        S = np.stack([synthetic.random_density(ad.n, seed=20 + r) for r in range(3)])
        d = torch.from_numpy(S.astype(np.complex64).reshape(-1)).cuda()
        o = torch.empty_like(d)
        ad.matvec(d, o, 3)
        torch.cuda.synchronize()
        got = o.cpu().numpy().astype(np.complex128).reshape(3, ad.n)
        for r in range(3):
            assert _rel(got[r], _mv(ad, S[r])) < 5e-6  # two runs differ by FP32 reduction order
    finally:
        ad.close()
        uni.close()
