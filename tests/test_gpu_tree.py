"""The octree and its lists, built by device kernels (Morton sort, leaf data,
neighbour lists, interaction lists bucketed by offset), against a numpy
restatement of their definitions (Sec. 2.3 octree and interaction lists; Sec.
3.1-3.2 Morton order):

  * the cube: side D = the power of two with D/2 < extent <= D, centred on the
    bounding box; a point's cell at level l is floor((x - lo) 2^l / D) (at most
    2^l - 1 per axis);
  * depth L: the smallest level whose fullest cell holds <= leaf_max points;
  * near field: leaf pairs within one cell in each coordinate (27-neighbourhood);
  * M2L at level l >= 2: source cells that are children of the target's parent's
    neighbours but not neighbours of the target;
  * M2M / L2L: one translation per (child, parent) pair.

Exact integer equality of every count.

Adaptive trees (config adaptive = 1): a box is split only while it holds more than
leaf_max points (or until the depth cap); leaves that touch interact directly (U); a box
that does not touch leaf t while its parent does, under a same-level neighbour of t, meets
t through M2P and P2L (W and its dual X); M2L runs between same-level boxes that do not
touch and whose parents do (V).  The restatement below builds the tree with dictionaries of
integer cells (no Morton keys) and finds the lists by brute force over all boxes, and checks
on its own lists that every ordered point pair is covered exactly once:
sum_U n_t n_s + sum_V |A| |B| + 2 sum_W n_t |c| = N^2 (W boxes with no more points than
expansion terms are summed directly, both ways, and count in U).
"""
import numpy as np
import pytest

import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _cells(X, leaf_max, depth=0):
    mn, mx = X.min(0), X.max(0)
    ext = float(np.max(mx - mn))
    D = 1.0
    if ext > 0:
        while D < ext:
            D *= 2.0
        while D * 0.5 >= ext:
            D *= 0.5
    lo = 0.5 * (mn + mx) - 0.5 * D
    q = np.clip(np.floor((X - lo) * (2.0 ** 20 / D)), 0, 2 ** 20 - 1).astype(np.int64)
    L = depth
    if L <= 0:
        for L in range(21):
            _, cnt = np.unique(q >> (20 - L), axis=0, return_counts=True)
            if cnt.max() <= leaf_max:
                break
    return [np.unique(q >> (20 - l), axis=0, return_counts=True) for l in range(L + 1)], L


def _enc(c):
    return (c[:, 0] << 42) | (c[:, 1] << 21) | c[:, 2]


def _lookup(cells, keys_sorted, order, cand, n_l):
    """Index (into cells) of each candidate cell, or -1."""
    ok = np.all((cand >= 0) & (cand < n_l), axis=1)
    e = _enc(np.where(ok[:, None], cand, 0))
    pos = np.clip(np.searchsorted(keys_sorted, e), 0, len(keys_sorted) - 1)
    hit = ok & (keys_sorted[pos] == e)
    return np.where(hit, order[pos], -1)


def _expected(X, leaf_max, orders_of, depth=0):
    lv, L = _cells(X, leaf_max, depth)
    out = {"depth": L, "n_leaves": len(lv[L][0])}
    # near field over the leaves
    leaf, nleaf = lv[L]
    ek = _enc(leaf)
    order = np.argsort(ek)
    ks = ek[order]
    pairs = 0
    for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T:
        j = _lookup(leaf, ks, order, leaf + d, 2 ** L)
        pairs += int(np.sum(np.where(j >= 0, nleaf * nleaf[np.maximum(j, 0)], 0)))
    out["near_pairs"] = pairs - X.shape[0]
    # M2L
    m2l, m2l_cmacs, trans = 0, 0, 0
    offs = np.array(np.meshgrid(*[np.arange(-3, 4)] * 3, indexing="ij")).reshape(3, -1).T
    offs = offs[np.max(np.abs(offs), axis=1) >= 2]
    for l in range(2, L + 1):
        c = lv[l][0]
        ek = _enc(c)
        order = np.argsort(ek)
        ks = ek[order]
        n = 0
        for d in offs:
            s = c + d
            par_ok = np.all(np.abs((s >> 1) - (c >> 1)) <= 1, axis=1)
            j = _lookup(c, ks, order, s, 2 ** l)
            n += int(np.sum(par_ok & (j >= 0)))
        m2l += n
        m2l_cmacs += n * orders_of(l) ** 2
        if l >= 3:  # M2M into level l-1 and L2L out of it: one per box of level l
            trans += 2 * len(c) * orders_of(l) * orders_of(l - 1)
    out["m2l"] = m2l
    out["m2l_cmacs"] = m2l_cmacs
    out["m2m_l2l_cmacs"] = trans
    # every ordered point pair exactly once: near leaf pairs plus M2L box pairs
    cover = 0
    for l in range(2, L + 1):
        c, n = lv[l]
        ek = _enc(c)
        order = np.argsort(ek)
        ks = ek[order]
        for d in offs:
            s_ = c + d
            par_ok = np.all(np.abs((s_ >> 1) - (c >> 1)) <= 1, axis=1)
            j = _lookup(c, ks, order, s_, 2 ** l)
            ok = par_ok & (j >= 0)
            cover += int(np.sum(n[ok] * n[j[ok]]))
    assert pairs + cover == X.shape[0] ** 2
    return out


CASES = [
    ("sphere_1280_leaf64", lambda: synthetic.sphere_mesh(3), 1.0, dict(p_fixed=8, leaf_max=64)),
    ("sphere_320_leaf10", lambda: synthetic.sphere_mesh(2), 3.0, dict(leaf_max=10)),
    ("ellipsoid_5120_leaf16", lambda: synthetic.ellipsoid_mesh(4), 5.0, dict(leaf_max=16)),
    ("star_8000", lambda: synthetic.serving_shape("star", 20, seed=3), 4.0, {}),
    ("sphere_5120_depth5", lambda: synthetic.sphere_mesh(4), 2.0, dict(depth=5)),
]


@pytest.mark.parametrize("name,mesh,k,kw", CASES, ids=[c[0] for c in CASES])
def test_tree_counts_match_definition(name, mesh, k, kw):
    V, F = mesh()
    plan = pkg.Plan(V, F, k, **kw)
    try:
        info, costs = plan.info(), plan.costs()
        X, _, _ = plan.points()
        P = lambda l: (info["orders"][l] + 1) ** 2  # noqa: E731
        exp = _expected(X, plan.cfg.leaf_max, P, depth=kw.get("depth", 0))
        assert info["depth"] == exp["depth"]
        assert info["n_leaves"] == exp["n_leaves"]
        assert info["m2l_translations"] == exp["m2l"]
        assert costs["p2p_pairs"] == exp["near_pairs"]
        assert costs["m2l_cmacs"] == exp["m2l_cmacs"]
        assert costs["m2m_l2l_cmacs"] == exp["m2m_l2l_cmacs"]
        assert costs["n_points"] == plan.n
    finally:
        plan.close()


def test_cube_face_points_are_clamped_into_the_last_cell():
    """A closed box surface: points on the upper faces sit at the cube's edge when the
    extent is a power of two; they fall into the last cell of each level."""
    V = np.array([[0, 0, 0], [4, 0, 0], [4, 4, 0], [0, 4, 0], [0, 0, 4], [4, 0, 4], [4, 4, 4], [0, 4, 4]], float)
    F = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4], [2, 3, 7], [2, 7, 6],
                  [1, 2, 6], [1, 6, 5], [0, 4, 7], [0, 7, 3]], dtype=np.int32)
    Vr, Fr = V, F
    for _ in range(6):
        Vr, Fr = synthetic.bisect_longest_edges(Vr, Fr)
    plan = pkg.Plan(Vr, Fr, 1.0, leaf_max=8)
    try:
        info, costs = plan.info(), plan.costs()
        X, _, _ = plan.points()
        P = lambda l: (info["orders"][l] + 1) ** 2  # noqa: E731
        exp = _expected(X, 8, P)
        assert (info["depth"], info["n_leaves"], info["m2l_translations"]) == (exp["depth"], exp["n_leaves"], exp["m2l"])
        assert costs["p2p_pairs"] == exp["near_pairs"] and costs["m2l_cmacs"] == exp["m2l_cmacs"]
    finally:
        plan.close()


def _adaptive_expected(X, leaf_max, orders_of, maxdepth=20):
    """The adaptive tree by brute force over its boxes: U(t) = the leaves touching leaf t;
    W(t) = the boxes that do not touch t, whose parents do, and that lie under a same-level
    neighbour of t (M2P to t and P2L from t), except that a W box holding no more points than
    its expansion has terms is summed directly both ways; V = same-level boxes that do not
    touch while their parents do (M2L).  Touching: closed boxes in level-20 units."""
    mn, mx = X.min(0), X.max(0)
    ext = float(np.max(mx - mn))
    D = 1.0
    if ext > 0:
        while D < ext:
            D *= 2.0
        while D * 0.5 >= ext:
            D *= 0.5
    lo = 0.5 * (mn + mx) - 0.5 * D
    q = np.clip(np.floor((X - lo) * (2.0 ** 20 / D)), 0, 2 ** 20 - 1).astype(np.int64)
    boxes = {}  # (level, cell) -> (point count, is leaf)
    stack = [(0, (0, 0, 0), np.arange(X.shape[0]))]
    while stack:
        l, c, idx = stack.pop()
        leaf = len(idx) <= leaf_max or l == maxdepth
        boxes[(l, c)] = (len(idx), leaf)
        if not leaf:
            ch = q[idx] >> (20 - (l + 1))
            keys, inv = np.unique(ch, axis=0, return_inverse=True)
            for j, kc in enumerate(keys):
                stack.append((l + 1, tuple(int(v) for v in kc), idx[inv.ravel() == j]))
    items = list(boxes.items())
    lev = np.array([l for (l, _), _ in items])
    cell = np.array([c for (_, c), _ in items], dtype=np.int64)
    npt = np.array([n for _, (n, _) in items], dtype=np.int64)
    isleaf = np.array([lf for _, (_, lf) in items])
    span = np.left_shift(1, 20 - lev)
    blo = cell * span[:, None]
    bhi = (cell + 1) * span[:, None]
    plo = (cell >> 1) * (2 * span)[:, None]
    phi_ = ((cell >> 1) + 1) * (2 * span)[:, None]

    def touch(lo1, hi1, lo2, hi2):
        return np.all((lo1 <= hi2) & (lo2 <= hi1), axis=-1)

    L = int(lev[isleaf].max())
    Pl = np.array([orders_of(int(l)) if l >= 2 else 0 for l in lev])
    near = wcov = 0
    for t in np.flatnonzero(isleaf):
        lt = lev[t]
        tu = touch(blo[t], bhi[t], blo, bhi)
        near += npt[t] * int(np.sum(npt[tu & isleaf]))
        deeper = lev > lt
        anc = cell >> np.maximum(lev - lt, 0)[:, None]
        under_nbr = deeper & np.all(np.abs(anc - cell[t]) <= 1, axis=1)
        w = under_nbr & ~tu & touch(blo[t], bhi[t], plo, phi_)
        small = w & (npt <= Pl)  # fewer points than expansion terms: direct, both ways
        near += 2 * npt[t] * int(np.sum(npt[small]))
        wcov += 2 * npt[t] * int(np.sum(npt[w & ~small]))
    m2l, cmacs, cover = 0, 0, 0
    offs = [(dx, dy, dz) for dx in range(-3, 4) for dy in range(-3, 4) for dz in range(-3, 4)
            if max(abs(dx), abs(dy), abs(dz)) >= 2]
    for (l, c), (n, _) in boxes.items():
        if l < 2:
            continue
        for d in offs:
            s_ = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
            if all(abs((s_[i] >> 1) - (c[i] >> 1)) <= 1 for i in range(3)) and (l, s_) in boxes:
                m2l += 1
                cmacs += orders_of(l) ** 2
                cover += n * boxes[(l, s_)][0]
    trans = sum(2 * orders_of(l) * orders_of(l - 1) for (l, _) in boxes if l >= 3)
    N = X.shape[0]
    assert near + cover + wcov == N * N  # every ordered pair exactly once (i = j counted as direct)
    return {"depth": L, "n_leaves": int(isleaf.sum()), "near_pairs": near - N, "m2l": m2l, "m2l_cmacs": cmacs,
            "m2m_l2l_cmacs": trans}


ADAPTIVE_CASES = [
    ("cap_sphere_5952_leaf32", lambda: synthetic.refined_cap_sphere(3, 4), 2.0, dict(leaf_max=32, p_fixed=6)),
    ("ellipsoid_5120_leaf16", lambda: synthetic.ellipsoid_mesh(4), 5.0, dict(leaf_max=16)),
    ("sphere_5120_leaf40", lambda: synthetic.sphere_mesh(4), 3.0, dict(leaf_max=40)),
    ("cap_sphere_depth_cap", lambda: synthetic.refined_cap_sphere(2, 5), 1.0, dict(leaf_max=8, depth=4)),
]


@pytest.mark.parametrize("name,mesh,k,kw", ADAPTIVE_CASES, ids=[c[0] for c in ADAPTIVE_CASES])
def test_adaptive_tree_counts_match_definition(name, mesh, k, kw):
    V, F = mesh()
    plan = pkg.Plan(V, F, k, adaptive=1, **kw)
    try:
        info, costs = plan.info(), plan.costs()
        X, _, _ = plan.points()
        P = lambda l: (info["orders"][l] + 1) ** 2  # noqa: E731
        exp = _adaptive_expected(X, plan.cfg.leaf_max, P, maxdepth=kw.get("depth", 0) or 20)
        assert info["depth"] == exp["depth"]
        assert info["n_leaves"] == exp["n_leaves"]
        assert info["m2l_translations"] == exp["m2l"]
        assert costs["p2p_pairs"] == exp["near_pairs"]
        assert costs["m2l_cmacs"] == exp["m2l_cmacs"]
        assert costs["m2m_l2l_cmacs"] == exp["m2m_l2l_cmacs"]
    finally:
        plan.close()
