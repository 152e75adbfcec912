"""Closed triangulated surfaces used as synthetic scatterers.

The paper's experiments scatter a plane wave off a sphere of radius 1 m meshed
with curvilinear triangles (Sec. 5.2, Table "Mesh dataset descriptions"); those
meshes are not available, so flat-triangle icospheres stand in for them.

Every mesh is returned as ``(V, F)``: ``V`` float64 [n_vert, 3] vertex
coordinates and ``F`` int32 [n_tri, 3] vertex indices, counter-clockwise seen
from outside.  Nothing here depends on a random state except ``star_mesh``,
which takes an explicit seed.
"""
from __future__ import annotations

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron():
    v = np.array(
        [
            [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
            [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
            [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def _split4(v, f):
    """One 1-to-4 refinement; new edge midpoints are pushed onto the unit sphere."""
    nv = v.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
    uniq, inv = np.unique(key, return_inverse=True)
    a = uniq // nv
    b = uniq % nv
    mid = 0.5 * (v[a] + v[b])
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    nt = f.shape[0]
    m01 = nv + inv[:nt]
    m12 = nv + inv[nt:2 * nt]
    m20 = nv + inv[2 * nt:]
    f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
    nf = np.concatenate(
        [
            np.stack([f0, m01, m20], 1),
            np.stack([m01, f1, m12], 1),
            np.stack([m20, m12, f2], 1),
            np.stack([m01, m12, m20], 1),
        ],
        axis=0,
    )
    return np.concatenate([v, mid], axis=0), nf


def icosphere(level: int):
    """Unit-sphere icosphere with 20 * 4**level triangles."""
    v, f = _icosahedron()
    for _ in range(level):
        v, f = _split4(v, f)
    return v, f.astype(np.int32)


def bisect_longest_edges(v, f):
    """Split every triangle in two across its longest edge.

    The new vertex is the midpoint of that edge and is NOT moved onto the
    sphere, so the refined mesh covers exactly the same polyhedral surface
    (a neighbour that split a different edge sees a T-junction, which a
    Nystrom discretisation with interior points does not mind).  Ties between
    equal edge lengths go to the lowest edge slot (0: v0-v1, 1: v1-v2, 2: v2-v0).
    """
    f = np.asarray(f, dtype=np.int64)
    p0, p1, p2 = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    l = np.stack(
        [
            np.sum((p1 - p0) ** 2, axis=1),
            np.sum((p2 - p1) ** 2, axis=1),
            np.sum((p0 - p2) ** 2, axis=1),
        ],
        axis=1,
    )
    s = np.argmax(l, axis=1)  # first maximum wins ties
    # rotate each triangle so that its longest edge is (a, b), apex c
    a = np.where(s == 0, f[:, 0], np.where(s == 1, f[:, 1], f[:, 2]))
    b = np.where(s == 0, f[:, 1], np.where(s == 1, f[:, 2], f[:, 0]))
    c = np.where(s == 0, f[:, 2], np.where(s == 1, f[:, 0], f[:, 1]))
    # an edge shared by two triangles that both split it gets one midpoint
    nv = v.shape[0]
    key = np.minimum(a, b) * nv + np.maximum(a, b)
    uniq, inv = np.unique(key, return_inverse=True)
    ua, ub = uniq // nv, uniq % nv
    mid = 0.5 * (v[ua] + v[ub])
    m = nv + inv
    nf = np.empty((2 * f.shape[0], 3), dtype=np.int64)
    nf[0::2] = np.stack([a, m, c], 1)
    nf[1::2] = np.stack([m, b, c], 1)
    return np.concatenate([v, mid], axis=0), nf.astype(np.int32)


def refined_cap_sphere(level: int, extra: int, z0: float = 0.5):
    """Icosphere of the given level whose triangles with centroid z > z0 are split across
    their longest edge `extra` more times (T-junctions at the cap's rim): the point density
    in the cap is 2^extra times the rest, the non-uniform case for an adaptive octree."""
    v, f = icosphere(level)
    for _ in range(extra):
        c = (v[f[:, 0]] + v[f[:, 1]] + v[f[:, 2]]) / 3.0
        cap = c[:, 2] > z0
        v2, f2 = bisect_longest_edges(v, f[cap])
        v, f = v2, np.concatenate([f[~cap], f2]).astype(np.int32)
    return v, f


def sphere_mesh(level: int, bisect: bool = False, radius: float = 1.0):
    v, f = icosphere(level)
    if bisect:
        v, f = bisect_longest_edges(v, f)
    return v * radius, f


def ellipsoid_mesh(level: int, axes=(2.0, 1.0, 1.0), bisect: bool = False):
    v, f = sphere_mesh(level, bisect)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


def star_mesh(level: int, seed: int, amplitude: float = 0.2):
    """Star-shaped surface r(x) = 1 + amplitude * S(x) / max|S| on an icosphere.

    S is a seeded random combination of the monomials x^a y^b z^c with
    1 <= a+b+c <= 3 restricted to the unit sphere, i.e. a random function in
    the span of the spherical harmonics of degree 1..3.
    """
    v, f = icosphere(level)
    rng = np.random.default_rng(seed)
    exps = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if 1 <= a + b + c <= 3]
    coef = rng.standard_normal(len(exps))
    s = np.zeros(v.shape[0])
    for w, (a, b, c) in zip(coef, exps):
        s += w * v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c
    s /= np.max(np.abs(s))
    return v * (1.0 + amplitude * s)[:, None], f


def triangle_soup(n_tri: int, seed: int, size: float = 0.02, extent: float = 0.99):
    """n_tri small random triangles (edges about `size`) with centres uniform in the
    cube [-extent, extent]^3: points fill a volume, so the leaves of an octree over
    them are full and neighbouring leaves meet at every relative position."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, (n_tri, 3))
    v = c[:, None, :] + size * rng.standard_normal((n_tri, 3, 3))
    f = np.arange(3 * n_tri, dtype=np.int64).reshape(n_tri, 3)
    return v.reshape(-1, 3), f


def corner_lattice_soup(cells: int, margin: float, seed: int, size: float = 3e-4):
    """Tiny random triangles centred near the 8 corners of every cell of a
    cells^3 grid over [-1, 1]^3 (a fraction `margin` of the cell side inside
    each corner): points of neighbouring cells then sit at every relative
    position up to the far corners of a 2 x 2 x 2 block of cells."""
    rng = np.random.default_rng(seed)
    h = 2.0 / cells
    one = np.array([margin, 1.0 - margin]) * h
    base = -1.0 + h * np.arange(cells)
    ax = (base[:, None] + one[None, :]).ravel()
    c = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    v = c[:, None, :] + size * rng.standard_normal((c.shape[0], 3, 3))
    f = np.arange(3 * c.shape[0], dtype=np.int64).reshape(-1, 3)
    return v.reshape(-1, 3), f


def geodesic_sphere(nu: int):
    """Unit sphere from the icosahedron with every face cut into nu^2 triangles
    (geodesic frequency nu): 20 nu^2 triangles, 10 nu^2 + 2 vertices."""
    if nu < 1:
        raise ValueError("frequency must be at least 1")
    v0, f0 = _icosahedron()
    # barycentric grid of one face: (i, j) with i + j <= nu
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nu + 1), indexing="ij")
    keep = ii + jj <= nu
    ii, jj = ii[keep], jj[keep]
    lid = -np.ones((nu + 1, nu + 1), dtype=np.int64)
    lid[ii, jj] = np.arange(ii.size)
    up = [(i, j) for i in range(nu) for j in range(nu - i)]
    dn = [(i, j) for i in range(nu) for j in range(nu - i - 1)]
    tri_local = np.array([[lid[i, j], lid[i + 1, j], lid[i, j + 1]] for i, j in up]
                         + [[lid[i + 1, j], lid[i + 1, j + 1], lid[i, j + 1]] for i, j in dn], dtype=np.int64)
    verts, faces = [], []
    for a, b, c in f0:
        p = (v0[a][None, :] * (nu - ii - jj)[:, None] + v0[b][None, :] * ii[:, None]
             + v0[c][None, :] * jj[:, None]) / nu
        faces.append(tri_local + sum(x.shape[0] for x in verts))
        verts.append(p)
    v = np.concatenate(verts, axis=0)
    f = np.concatenate(faces, axis=0)
    # points on shared edges appear once per face: merge them (exact grid positions)
    key = np.round(v * (8 * nu), 0).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    v = v[first]
    f = inv.reshape(-1)[f]
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f.astype(np.int32)


def serving_shape(kind: str, nu: int, seed: int, amplitude: float = 0.2):
    """A request's scatterer: 'sphere', 'ellipsoid' (semi-axes 2, 1, 1) or 'star'
    (r = 1 + amplitude S / max|S|, S a seeded degree-1..3 function as in star_mesh),
    on a geodesic mesh of frequency nu (N = 60 nu^2 quadrature points)."""
    v, f = geodesic_sphere(nu)
    if kind == "sphere":
        return v, f
    if kind == "ellipsoid":
        return v * np.array([2.0, 1.0, 1.0]), f
    if kind == "star":
        rng = np.random.default_rng(seed)
        exps = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if 1 <= a + b + c <= 3]
        coef = rng.standard_normal(len(exps))
        s = np.zeros(v.shape[0])
        for w, (a, b, c) in zip(coef, exps):
            s += w * v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c
        s /= np.max(np.abs(s))
        return v * (1.0 + amplitude * s)[:, None], f
    raise ValueError(f"unknown shape {kind!r}")


def serving_requests(n: int, seed: int = 0, rate: float = 20.0, n_min: int = 10_000, n_max: int = 1_000_000,
                     k_range=(1.0, 30.0), nrhs_max: int = 16):
    """n request specifications for the serving workload: Poisson arrivals at `rate`
    per second, shape uniform over sphere / ellipsoid / star, N log-uniform in
    [n_min, n_max] (rounded to a geodesic frequency, N = 60 nu^2), k uniform in
    k_range, 1..nrhs_max right-hand sides (incident directions seeded per request)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    shapes = ["sphere", "ellipsoid", "star"]
    out = []
    for q in range(n):
        target = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        nu = max(1, int(round((target / 60.0) ** 0.5)))
        out.append({"id": q, "arrival_s": float(t[q]), "shape": shapes[int(rng.integers(3))], "nu": nu,
                    "n_points": 60 * nu * nu, "k": float(rng.uniform(*k_range)),
                    "nrhs": int(rng.integers(1, nrhs_max + 1)), "seed": int(rng.integers(2 ** 31))})
    return out


# Named workloads: (description, builder).  Triangle counts follow the
# configurations the benchmarks and parity tests use.
WORKLOADS = {
    # 20 * 4**3 = 1,280 triangles -> N = 3,840 points
    "sphere_1280": ("unit sphere, icosphere level 3", lambda: sphere_mesh(3)),
    # 20 * 4**5 * 2 = 40,960 triangles -> N = 122,880 points (small batched case for profiling)
    "sphere_40960": ("unit sphere, icosphere level 5 + longest-edge bisection", lambda: sphere_mesh(5, True)),
    # 20 * 4**6 * 2 = 163,840 triangles -> N = 491,520 points
    "sphere_163840": ("unit sphere, icosphere level 6 + longest-edge bisection", lambda: sphere_mesh(6, True)),
    # 20 * 4**7 * 2 = 655,360 triangles -> N = 1,966,080 points
    "sphere_655360": ("unit sphere, icosphere level 7 + longest-edge bisection", lambda: sphere_mesh(7, True)),
    # 20 * 4**8 = 1,310,720 triangles -> N = 3,932,160 points
    "ellipsoid_1310720": ("ellipsoid (2,1,1), icosphere level 8", lambda: ellipsoid_mesh(8)),
    # icosphere level 6 with the cap z > 0.5 bisected 4 more times (16x the point density):
    # 387,864 triangles -> N = 1,163,592 points, the non-uniform case for the adaptive tree
    "cap_sphere_387864": ("unit sphere, icosphere level 6, cap z > 0.5 refined 4 more times",
                         lambda: refined_cap_sphere(6, 4)),
}


def workload_mesh(name: str):
    return WORKLOADS[name][1]()
