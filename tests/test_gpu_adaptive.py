"""Adaptive octree (config adaptive = 1) through the C ABI on a sphere whose cap carries 16
times the point density of the rest (leaves at two to three depths; the far field uses the
M2L, M2P and P2L lists):

  matvec vs the oracle's FP64 direct sum on sampled rows      1e-4  (p = 8 and 10: the fixed-
                                                                     order and any-order P2M/L2P)
  adaptive vs uniform plan, same orders                         1e-4
  near field alone vs the oracle's point sum over the         1e-5  (FP32 P2P; the direct pairs
  target's direct leaves (restated from the definition)               are exactly these)
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


def _tree(X, leaf_max):
    """The adaptive tree from its definition (a box splits while it holds more than leaf_max
    points): every box (level, cell, point count, leaf id or -1) and each point's leaf."""
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
    lev, cell, npt, lid = [], [], [], []
    nleaf = 0
    stack = [(0, np.arange(X.shape[0]))]
    while stack:
        l, idx = stack.pop()
        lev.append(l)
        cell.append(q[idx[0]] >> (20 - l))
        npt.append(len(idx))
        if len(idx) <= leaf_max:
            leaf_of[idx] = nleaf
            lid.append(nleaf)
            nleaf += 1
            continue
        lid.append(-1)
        ch = q[idx] >> (20 - (l + 1))
        keys, inv = np.unique(ch, axis=0, return_inverse=True)
        for j in range(len(keys)):
            stack.append((l + 1, idx[inv.ravel() == j]))
    return leaf_of, np.array(lev), np.array(cell), np.array(npt), np.array(lid)


def test_adaptive_near_field_against_point_sum(cap):
    """parts = 1 (near field only): every target against the points of its direct leaves, i.e.
    the leaves that touch its leaf t, the leaves under t's W boxes that hold no more points
    than expansion terms, and the leaves s with such a W box containing t; against the
    oracle's point sum over exactly those sources (sampled targets)."""
    V, F, k = cap
    plan = pkg.Plan(V, F, k, adaptive=1, leaf_max=32, p_fixed=8)
    try:
        X, W, _ = plan.points()
        Pn = 81  # (p + 1)^2 on every level
        s = synthetic.random_density(plan.n, seed=7)
        got = _mv(plan, s, parts=1)
        leaf_of, lev, cell, npt, lid = _tree(X, 32)
        assert plan.info()["n_leaves"] == int((lid >= 0).sum())
        span = np.left_shift(1, 20 - lev)
        blo, bhi = cell * span[:, None], (cell + 1) * span[:, None]
        plo, phi_ = (cell >> 1) * (2 * span)[:, None], ((cell >> 1) + 1) * (2 * span)[:, None]
        leafbox = np.full(int((lid >= 0).sum()), -1)
        leafbox[lid[lid >= 0]] = np.flatnonzero(lid >= 0)

        def touch(a, b, lo_, hi_):
            return np.all((a <= hi_) & (lo_ <= b), axis=-1)

        def small_w(tb):  # boxes that are small W boxes of the leaf in box tb
            deeper = lev > lev[tb]
            anc = cell >> np.maximum(lev - lev[tb], 0)[:, None]
            under = deeper & np.all(np.abs(anc - cell[tb]) <= 1, axis=1)
            w = under & ~touch(blo[tb], bhi[tb], blo, bhi) & touch(blo[tb], bhi[tb], plo, phi_)
            return w & (npt <= Pn)

        def inside(outer, inner):  # box inner within box outer
            return np.all((blo[outer] <= blo[inner]) & (bhi[inner] <= bhi[outer]), axis=-1)

        rng = np.random.default_rng(11)
        for i in rng.choice(plan.n, 40, replace=False):
            tb = leafbox[leaf_of[i]]
            direct = set(lid[(lid >= 0) & touch(blo[tb], bhi[tb], blo, bhi)])
            for c in np.flatnonzero(small_w(tb)):  # leaves under t's small W boxes
                direct |= set(lid[(lid >= 0) & inside(c, np.arange(len(lev)))])
            for sb in np.flatnonzero((lid >= 0) & (lev < lev[tb])):  # t under a small W box of s
                if np.any(small_w(sb) & inside(np.arange(len(lev)), tb)):
                    direct.add(lid[sb])
            src = np.flatnonzero(np.isin(leaf_of, list(direct)))
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
