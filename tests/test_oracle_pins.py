"""Pins of the FP64 oracle against facts fixed by mathematics or the paper.

Every check here is independent of the oracle's own formulas: closed forms,
library special functions, brute-force quadrature written here in numpy,
symmetry, additivity, spectral facts of the sphere and convergence rates.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.special import eval_legendre, sph_harm_y, spherical_jn, spherical_yn

import oracle
import synthetic

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------- helpers
def _polar_bruteforce(x, v, k, n=160):
    """int_T G(x,y) L_a(y) dS for x in the plane of T (inside T), in polar
    coordinates about x: the integrand rho*G*L is smooth there, so tensor
    Gauss-Legendre converges without any singular treatment."""
    v = np.asarray(v, dtype=float).reshape(3, 3)
    e1, e2 = v[1] - v[0], v[2] - v[0]
    nrm = np.cross(e1, e2)
    A2 = np.linalg.norm(nrm)
    nh = nrm / A2
    grads = np.array([np.cross(nh, v[(a + 2) % 3] - v[(a + 1) % 3]) / A2 for a in range(3)])
    g, w = leggauss(n)
    g, w = (g + 1) / 2, w / 2
    U, Tt = np.meshgrid(g, g, indexing="ij")
    WW = np.outer(w, w)
    out = np.zeros(3, complex)
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        # sub-triangle (x, a, b): y = x + t*(a + u*(b-a) - x), dS = t*|(a-x) x (b-a)|
        jac = np.linalg.norm(np.cross(a - x, b - a))
        E = a[None, None] + U[..., None] * (b - a)[None, None] - x[None, None]
        En = np.linalg.norm(E, axis=-1)
        y = x[None, None] + Tt[..., None] * E
        f = np.exp(1j * k * Tt * En) / (4 * np.pi * En) * jac * WW  # t * G * jacobian
        lam = (y - v[0]) @ grads.T
        lam[..., 0] += 1.0
        out += np.einsum("ij,ijq->q", f, 2 * lam - 1 / 3)
    return out


def _subdivided_rule(x, v, k, n=20, depth=3):
    """Smooth-integrand brute force: conical Gauss on 4**depth sub-triangles."""
    v = np.asarray(v, dtype=float).reshape(3, 3)
    tris = [v]
    for _ in range(depth):
        nt = []
        for t in tris:
            m01, m12, m20 = (t[0] + t[1]) / 2, (t[1] + t[2]) / 2, (t[2] + t[0]) / 2
            nt += [np.array([t[0], m01, m20]), np.array([m01, t[1], m12]),
                   np.array([m20, m12, t[2]]), np.array([m01, m12, m20])]
        tris = nt
    g, w = leggauss(n)
    g, w = (g + 1) / 2, w / 2
    U, Vv = np.meshgrid(g, g, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    s, t, ww = U.ravel(), (Vv * (1 - U)).ravel(), (WU * WV * (1 - U)).ravel()
    e1, e2 = v[1] - v[0], v[2] - v[0]
    nrm = np.cross(e1, e2)
    A2 = np.linalg.norm(nrm)
    nh = nrm / A2
    grads = [np.cross(nh, v[(a + 2) % 3] - v[(a + 1) % 3]) / A2 for a in range(3)]
    out = np.zeros(3, complex)
    for T in tris:
        f1, f2 = T[1] - T[0], T[2] - T[0]
        a2 = np.linalg.norm(np.cross(f1, f2))
        y = T[0][None] + s[:, None] * f1[None] + t[:, None] * f2[None]
        R = np.linalg.norm(x[None] - y, axis=1)
        G = np.exp(1j * k * R) / (4 * np.pi * R)
        for a in range(3):
            lam = (1.0 if a == 0 else 0.0) + (y - v[0]) @ grads[a]
            out[a] += np.sum(ww * a2 * G * (2 * lam - 1 / 3))
    return out


def _split4(v):
    v = np.asarray(v, dtype=float).reshape(3, 3)
    m01, m12, m20 = (v[0] + v[1]) / 2, (v[1] + v[2]) / 2, (v[2] + v[0]) / 2
    return [np.array([v[0], m01, m20]), np.array([m01, v[1], m12]),
            np.array([m20, m12, v[2]]), np.array([m01, m12, m20])]


# ---------------------------------------------------------------- special functions
def test_spherical_bessel_against_scipy():
    n = np.arange(21)
    for z in [1e-3, 0.3, 1.7, 2.3, 8.66, 31.0]:
        assert np.allclose(oracle.sph_jn(20, z), spherical_jn(n, z), rtol=1e-12, atol=1e-300)
        assert np.allclose(oracle.sph_yn(20, z), spherical_yn(n, z), rtol=1e-12)


def test_spherical_harmonics_against_scipy():
    # oracle: Y_n^{-m} = conj(Y_n^m); scipy: Y_n^{-m} = (-1)^m conj(Y_n^m)
    for th, ph in [(0.3, 2.1), (1.9, -0.4), (3.0, 5.5)]:
        Y = oracle.ylm(10, th, ph)
        for nn in range(11):
            for m in range(-nn, nn + 1):
                ref = sph_harm_y(nn, m, th, ph) * ((-1) ** m if m < 0 else 1)
                assert abs(Y[nn * nn + nn + m] - ref) < 1e-13


def test_addition_theorem_reproduces_green():
    """G(x,y) = i k sum_n j_n(k|y|) h_n(k|x|) sum_m Y_nm(x^) conj(Y_nm(y^)), |y| < |x|,
    assembled from the oracle's special functions at p = 30 (the convention
    behind every expansion of the FMM)."""
    k = 3.0
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = rng.standard_normal(3)
        x *= 1.5 / np.linalg.norm(x)
        y = rng.standard_normal(3)
        y *= 0.4 / np.linalg.norm(y)
        rx, ry = np.linalg.norm(x), np.linalg.norm(y)
        tx, px = np.arccos(x[2] / rx), np.arctan2(x[1], x[0])
        ty, py = np.arccos(y[2] / ry), np.arctan2(y[1], y[0])
        p = 30
        jn, hn = oracle.sph_jn(p, k * ry), oracle.sph_jn(p, k * rx) + 1j * oracle.sph_yn(p, k * rx)
        Yx, Yy = oracle.ylm(p, tx, px), oracle.ylm(p, ty, py)
        s = 0j
        for nn in range(p + 1):
            sl = slice(nn * nn, (nn + 1) ** 2)
            s += jn[nn] * hn[nn] * np.sum(Yx[sl] * np.conj(Yy[sl]))
        R = np.linalg.norm(x - y)
        assert abs(1j * k * s - np.exp(1j * k * R) / (4 * np.pi * R)) < 1e-12


# ---------------------------------------------------------------- singular integrals
def test_one_over_R_equilateral_centroid_closed_form():
    # polar coordinates about the centroid: 3 * int_{-pi/3}^{pi/3} d/cos(phi) dphi,
    # d = s/(2 sqrt 3)  ->  sqrt(3) s ln(2 + sqrt 3)
    for s in [0.3, 1.0, 2.5]:
        v = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * np.sqrt(3) / 2, 0]])
        I0, I1 = oracle.tri_potential_1overR(v.mean(0), v)
        assert abs(I0 - np.sqrt(3) * s * np.log(2 + np.sqrt(3))) < 1e-14 * s
        assert np.linalg.norm(I1) < 1e-14 * s * s
        # k = 0: the three basis moments are equal by symmetry and sum to I0/(4 pi)
        t = oracle.tri_integrals(v.mean(0), v, 0.0)
        assert np.allclose(t, I0 / (3 * 4 * np.pi), rtol=1e-13)


@pytest.mark.parametrize("where", ["inside", "outside_inplane", "above", "far"])
def test_one_over_R_is_additive(where):
    rng = np.random.default_rng(7)
    v = rng.standard_normal((3, 3))
    c = v.mean(0)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    x = {"inside": 0.6 * v[0] + 0.3 * v[1] + 0.1 * v[2],
         "outside_inplane": 1.4 * v[0] - 0.2 * v[1] - 0.2 * v[2],
         "above": c + 0.05 * nrm + 0.1 * (v[1] - v[0]),
         "far": c + 5.0 * nrm}[where]
    I0, I1 = oracle.tri_potential_1overR(x, v)
    s0, s1 = 0.0, np.zeros(3)
    for ch in _split4(v):
        a0, a1 = oracle.tri_potential_1overR(x, ch)
        # I1 is taken about the same projection point for every child (same plane)
        s0, s1 = s0 + a0, s1 + a1
    assert abs(I0 - s0) < 1e-12 * abs(I0)
    assert np.linalg.norm(I1 - s1) < 1e-12 * max(np.linalg.norm(I1), abs(I0))


@pytest.mark.parametrize("k", [0.0, 2.0, 20.0])
def test_tri_integrals_offplane_against_bruteforce(k):
    rng = np.random.default_rng(3)
    v = rng.standard_normal((3, 3)) * 0.2
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    for x in [v.mean(0) + 0.05 * nrm, v[0] + 0.03 * nrm + 0.02 * (v[0] - v[1]), v.mean(0) + 2.0 * nrm]:
        a = oracle.tri_integrals(x, v, k)
        b = _subdivided_rule(x, v, k)
        assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b))


@pytest.mark.parametrize("k", [1.0, 10.0, 30.0])
def test_tri_integrals_self_against_polar_bruteforce(k):
    s = 0.25
    v = np.array([[0.0, 0.0, 0.0], [s, 0.02, 0.0], [0.4 * s, 0.9 * s, 0.0]])
    for bary in [(2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (0.45, 0.45, 0.1)]:
        x = bary[0] * v[0] + bary[1] * v[1] + bary[2] * v[2]
        a = oracle.tri_integrals(x, v, k)
        b = _polar_bruteforce(x, v, k)
        assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b))


def test_far_target_reduces_to_point_rule():
    """Far from a small triangle the exact basis moments approach the 3-point
    rule w G(x, x_a).  The rule integrates G L_a exactly up to its degree-2 part
    (this needs L_a(x_b) = delta_ab and w = A/3), so at low k the error falls
    as (h/d)^2."""
    v = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.03, 0.09, 0.0]])
    X, W, _ = oracle.points(v, np.array([[0, 1, 2]]))
    errs = []
    for d in [0.25, 0.5, 1.0]:
        x = np.array([0.04, 0.03, d])
        exact = oracle.tri_integrals(x, v, 0.01)
        R = np.linalg.norm(X - x, axis=1)
        pt = W * np.exp(0.01j * R) / (4 * np.pi * R)
        errs.append(np.max(np.abs(exact - pt)) / np.max(np.abs(pt)))
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


# ---------------------------------------------------------------- discretisation
def test_points_weights_cover_surface():
    V, F = synthetic.sphere_mesh(2)
    X, W, T = oracle.points(V, F)
    p = V[F]
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1).sum()
    assert abs(W.sum() - area) < 1e-12 * area
    assert np.all(T == np.repeat(np.arange(F.shape[0]), 3))
    # point a of triangle n: barycentric (2/3, 1/6, 1/6) rotated to vertex a
    n = 17
    assert np.allclose(X[3 * n + 1], (2 / 3) * p[n, 1] + (p[n, 0] + p[n, 2]) / 6)


def _mean_edge_numpy(V, F):
    V, F = np.asarray(V, float), np.asarray(F)
    L = [np.linalg.norm(V[F[:, (a + 1) % 3]] - V[F[:, a]], axis=1) for a in range(3)]
    return np.concatenate(L).mean()


@pytest.mark.parametrize("mesh", ["sphere", "star", "ellipsoid", "bisected"])
def test_mean_edge_against_numpy(mesh):
    """h-bar (the unit of the near radius, Sec. 6.4's near-patch distance) is the
    mean over all triangles of their three edge lengths."""
    V, F = {"sphere": lambda: synthetic.sphere_mesh(2),
            "star": lambda: synthetic.star_mesh(2, seed=3),
            "ellipsoid": lambda: synthetic.ellipsoid_mesh(2),
            "bisected": lambda: synthetic.sphere_mesh(2, bisect=True)}[mesh]()
    # sequential vs pairwise summation of ~2k terms: rounding well below 1e-12
    assert abs(oracle.mean_edge(V, F) - _mean_edge_numpy(V, F)) < 1e-12 * _mean_edge_numpy(V, F)
    # hand value: one right triangle with legs 3, 4 (edges 3, 4, 5)
    V1 = np.array([[0.0, 0, 0], [3.0, 0, 0], [0.0, 4, 0]])
    assert oracle.mean_edge(V1, np.array([[0, 1, 2]])) == 4.0


def _near_sets_bruteforce(X, T, r):
    """S(i) = {own triangle} U {triangle of every point j with |x_i - x_j| <= r}, squared
    distances summed in the same order (x, y, z) as any FP64 implementation would."""
    out = []
    r2 = r * r
    for i in range(X.shape[0]):
        d = X[i][None, :] - X
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        out.append(np.union1d([T[i]], T[d2 <= r2]))
    return out


@pytest.mark.parametrize("mesh,factor", [("sphere", 1.0), ("sphere", 2.5), ("star", 1.0), ("star", 1.7),
                                         ("bisected", 1.0)])
def test_near_sets_against_bruteforce(mesh, factor):
    """Sec. 2.2 / Listing 1: the own patch and every patch with a point within the near
    distance are integrated exactly; the oracle's hash-grid search must return exactly
    the brute-force set for every point."""
    V, F = {"sphere": lambda: synthetic.sphere_mesh(2),
            "star": lambda: synthetic.star_mesh(2, seed=5),
            "bisected": lambda: synthetic.sphere_mesh(1, bisect=True)}[mesh]()
    X, _, T = oracle.points(V, F)
    r = factor * _mean_edge_numpy(V, F)
    ptr, idx = oracle.near_sets(V, F, r)
    ref = _near_sets_bruteforce(X, T, r)
    sizes = np.diff(ptr)
    assert np.array_equal(sizes, [len(s) for s in ref])
    for i in range(X.shape[0]):
        assert np.array_equal(idx[ptr[i]:ptr[i + 1]], ref[i]), i
    # the sets are not trivially the own triangle: neighbours are found
    assert sizes.mean() > 4


def test_near_set_boundary_is_inclusive():
    """A triangle whose nearest point lies exactly at r_near belongs to S(i); one ulp
    less and it does not."""
    V, F = synthetic.star_mesh(2, seed=7)
    X, _, T = oracle.points(V, F)
    rng = np.random.default_rng(11)
    checked = 0
    for i in rng.permutation(X.shape[0])[:400]:
        d = X[i][None, :] - X
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        other = T != T[i]
        # the triangle of the nearest foreign point, and its nearest point's distance
        j = np.flatnonzero(other)[np.argmin(d2[other])]
        d2min = d2[T == T[j]].min()
        r = float(np.sqrt(d2min))
        if r * r != d2min:
            continue
        # nothing else sits between (r - 1 ulp) and r
        if np.count_nonzero(d2 == d2min) != 1:
            continue
        ptr, idx = oracle.near_sets(V, F, r)
        assert T[j] in idx[ptr[i]:ptr[i + 1]]
        ptr, idx = oracle.near_sets(V, F, np.nextafter(r, 0.0))
        assert T[j] not in idx[ptr[i]:ptr[i + 1]]
        checked += 1
        if checked == 3:
            break
    assert checked == 3


def test_near_set_overflow_is_refused():
    """A near radius that puts more candidates in one set than the oracle's table holds
    raises instead of silently truncating S(i)."""
    V, F = synthetic.sphere_mesh(4)  # 15,360 points, all within 2.1 of each other
    with pytest.raises(oracle.NearSetOverflow):
        oracle.near_sets(V, F, 2.1)
    with pytest.raises(oracle.NearSetOverflow):
        oracle.direct_rows(V, F, 1.0, 2.1, [0, 1], np.ones(3 * F.shape[0], complex))
    with pytest.raises(oracle.NearSetOverflow):
        oracle.correction_csr(V, F, 1.0, 2.1)


def test_operator_row_from_pinned_parts():
    """One row of Z assembled from the brute-force near set, the (separately pinned) exact
    triangle integrals and the point rule elsewhere (Eq. 10 with Sec. 2.2's treatment)
    equals the oracle's dense Z and its row-by-row form."""
    V, F = synthetic.star_mesh(1, seed=2)
    X, W, T = oracle.points(V, F)
    k, r = 3.0, 1.5 * _mean_edge_numpy(V, F)
    Z = oracle.dense_Z(V, F, k, r)
    S = _near_sets_bruteforce(X, T, r)
    rng = np.random.default_rng(4)
    for i in rng.choice(X.shape[0], 6, replace=False):
        R = np.linalg.norm(X[i] - X, axis=1)
        row = np.where(R > 0, W * np.exp(1j * k * R) / (4 * np.pi * np.where(R > 0, R, 1.0)), 0.0)
        for n in S[i]:
            row[3 * n:3 * n + 3] = oracle.tri_integrals(X[i], V[F[n]], k)
        assert np.allclose(Z[i], row, rtol=0, atol=1e-13 * np.abs(row).max())
        e = np.zeros(X.shape[0], complex)
        e[rng.integers(X.shape[0])] = 1.0
        s = synthetic.random_density(X.shape[0], int(i))
        assert abs(oracle.direct_rows(V, F, k, r, [i], s)[0] - row @ s) < 1e-12 * np.abs(row @ s)


def test_green_kernel_symmetry():
    V, F = synthetic.sphere_mesh(2)
    X, _, _ = oracle.points(V, F)
    one = np.ones(X.shape[0])
    u = synthetic.random_density(X.shape[0], 1)
    v = synthetic.random_density(X.shape[0], 2)
    Ku = oracle.point_sum(X, one, 2.5, u)
    Kv = oracle.point_sum(X, one, 2.5, v)
    assert abs(v @ Ku - u @ Kv) < 1e-12 * abs(v @ Ku)


def test_point_sum_rows_brute_force():
    """Sampled rows of the raw kernel sum against a numpy double loop written here."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((300, 3))
    X[7] = X[3]  # a coincident pair: R = 0 is skipped
    W = rng.uniform(0.5, 1.5, 300)
    s = synthetic.random_density(300, 9)
    rows = np.array([0, 3, 7, 150, 299])
    got = oracle.point_sum_rows(X, W, 4.0, s, rows)
    for q, i in enumerate(rows):
        acc = 0j
        for j in range(300):
            R = np.sqrt(((X[i] - X[j]) ** 2).sum())
            if j != i and R > 0:
                acc += W[j] * np.exp(4j * R) / (4 * np.pi * R) * s[j]
        assert abs(got[q] - acc) < 1e-13 * abs(acc)
    assert np.allclose(oracle.point_sum(X, W, 4.0, s)[rows], got, rtol=1e-14, atol=0)


def test_operator_forms_agree():
    """dense Z, the row-by-row definition, and point part + sparse correction."""
    V, F = synthetic.sphere_mesh(1)
    X, W, _ = oracle.points(V, F)
    k, r = 2.0, oracle.near_radius(V, F, 1.0)
    s = synthetic.random_density(X.shape[0], 5)
    Z = oracle.dense_Z(V, F, k, r)
    a = Z @ s
    b = oracle.direct_matvec(V, F, k, r, s)
    c = oracle.point_sum(X, W, k, s) + oracle.correction_csr(V, F, k, r) @ s
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)
    assert np.linalg.norm(a - c) < 1e-12 * np.linalg.norm(a)


def _eigen_errors(k, levels, n_list):
    out = {}
    for lev in levels:
        V, F = synthetic.sphere_mesh(lev)
        X, W, _ = oracle.points(V, F)
        r = oracle.near_radius(V, F, 1.0)
        ct = X[:, 2] / np.linalg.norm(X, axis=1)
        for nn in n_list:
            f = eval_legendre(nn, ct)
            if k == 0.0:
                lam = 1.0 / (2 * nn + 1)
            else:
                lam = 1j * k * spherical_jn(nn, k) * (spherical_jn(nn, k) + 1j * spherical_yn(nn, k))
            zf = oracle.direct_matvec(V, F, k, r, f)
            out[(lev, nn)] = np.linalg.norm(zf - lam * f) / np.linalg.norm(lam * f)
    return out


def test_laplace_limit_sphere_eigenvalues():
    """k -> 0: the single-layer operator on the unit sphere maps P_n(cos t) to P_n/(2n+1)."""
    e = _eigen_errors(0.0, [2, 3], [0, 1, 2, 3])
    for nn in [0, 1, 2, 3]:
        assert e[(3, nn)] < 0.02
        assert e[(3, nn)] < e[(2, nn)] / 2.5  # ~O(h^2) discretisation error


def test_helmholtz_sphere_eigenvalues():
    """P_n is an eigenfunction with eigenvalue i k j_n(k) h_n(k) (unit sphere)."""
    e = _eigen_errors(2.0, [2, 3], [0, 1, 2])
    for nn in [0, 1, 2]:
        assert e[(3, nn)] < 0.02
        assert e[(3, nn)] < e[(2, nn)] / 2.5


# ---------------------------------------------------------------- FMM
def test_fmm_converges_geometrically_in_p():
    V, F = synthetic.sphere_mesh(3)
    X, W, _ = oracle.points(V, F)
    s = synthetic.random_density(X.shape[0], 0)
    ref = oracle.point_sum(X, W, 1.0, s)
    errs = []
    for p in [4, 6, 8]:
        out, info = oracle.fmm(X, W, 1.0, s, leaf_max=64, p_fixed=p)
        assert info[0] == 3
        errs.append(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3
    assert errs[2] < 3e-5


def test_fmm_parts_and_pure_near_field():
    V, F = synthetic.sphere_mesh(2)
    X, W, _ = oracle.points(V, F)
    s = synthetic.random_density(X.shape[0], 4)
    full, _ = oracle.fmm(X, W, 4.0, s, p_fixed=6)
    near, _ = oracle.fmm(X, W, 4.0, s, p_fixed=6, parts=1)
    far, _ = oracle.fmm(X, W, 4.0, s, p_fixed=6, parts=2)
    assert np.allclose(full, near + far, rtol=0, atol=1e-14 * np.abs(full).max())
    # one leaf holding every point: the near field is the whole sum
    allnear, info = oracle.fmm(X, W, 4.0, s, leaf_max=10 ** 6)
    assert info[0] == 0
    ref = oracle.point_sum(X, W, 4.0, s)
    assert np.linalg.norm(allnear - ref) < 1e-13 * np.linalg.norm(ref)


# ---------------------------------------------------------------- GMRES / solution
def test_gmres_matches_dense_lu():
    V, F = synthetic.sphere_mesh(1)
    X, _, _ = oracle.points(V, F)
    Z = oracle.dense_Z(V, F, 1.0, oracle.near_radius(V, F, 1.0))
    b = oracle.plane_wave(X, 1.0, (0, 0, 1))
    x_lu = oracle.dense_solve(Z, b)
    x, it, rr, hist = oracle.gmres(lambda v: Z @ v, b, restart=30, tol=1e-10, maxiter=2000)
    assert rr < 2e-10
    assert np.linalg.norm(x - x_lu) < 1e-7 * np.linalg.norm(x_lu)
    # recurrence residual tracks the true one at exit
    assert abs(hist[-1] - rr) < 1e-3 * rr + 1e-14


def test_full_gmres_terminates_in_n_steps():
    V, F = synthetic.icosphere(0)
    X, _, _ = oracle.points(V, F)
    Z = oracle.dense_Z(V, F, 1.5, oracle.near_radius(V, F, 1.0))
    b = synthetic.random_density(X.shape[0], 9)
    x, it, rr, _ = oracle.gmres(lambda v: Z @ v, b, restart=X.shape[0], tol=1e-11, maxiter=X.shape[0])
    assert it <= X.shape[0] and rr < 1e-10


def test_solution_converges_to_mie_series():
    errs = []
    for lev in [2, 3]:
        V, F = synthetic.sphere_mesh(lev)
        X, _, _ = oracle.points(V, F)
        Z = oracle.dense_Z(V, F, 1.0, oracle.near_radius(V, F, 1.0))
        q = oracle.dense_solve(Z, oracle.plane_wave(X, 1.0, (0, 0, 1)))
        qm = oracle.mie_surface_q(X, 1.0)
        errs.append(np.linalg.norm(q - qm) / np.linalg.norm(qm))
    assert errs[1] < 1e-2 and errs[1] < errs[0] / 2


def test_mie_scattered_cancels_the_incident_wave_on_the_sphere():
    """Sound-soft boundary condition: p_inc + p_s = 0 at r = a, for several k and directions."""
    rng = np.random.default_rng(3)
    for k in (0.5, 2.0, 7.0):
        U = rng.standard_normal((40, 3))
        U /= np.linalg.norm(U, axis=1, keepdims=True)
        d = np.array([0.3, -0.4, 0.866])
        d /= np.linalg.norm(d)
        ps = oracle.mie_scattered(1.5 * U, k, a=1.5, d=d)
        pinc = np.exp(1j * k * (1.5 * U) @ d)
        assert np.max(np.abs(ps + pinc)) < 1e-10


def test_mie_scattered_outgoing_at_large_distance():
    """Radiation condition: r p_s e^{-ikr} tends to a function of direction only."""
    U = np.array([[0.0, 0.6, 0.8]])
    k = 3.0
    f1 = oracle.mie_scattered(200.0 * U, k) * 200.0 * np.exp(-1j * k * 200.0)
    f2 = oracle.mie_scattered(400.0 * U, k) * 400.0 * np.exp(-1j * k * 400.0)
    assert abs(f1[0] - f2[0]) < 2e-2 * abs(f2[0])


def test_field_direct_single_source_and_reciprocity():
    """One source: the Green's function itself; two point sets: u_A(B) . s_B = u_B(A) . s_A."""
    k = 1.7
    X = np.array([[0.1, -0.2, 0.3]])
    T = np.array([[2.0, 1.0, -0.5], [0.0, 0.0, 4.0]])
    u = oracle.field_direct(X, [2.0], k, [0.5 - 0.25j], T)
    R = np.linalg.norm(T - X, axis=1)
    assert np.allclose(u, 2.0 * (0.5 - 0.25j) * np.exp(1j * k * R) / (4 * np.pi * R), rtol=1e-14)
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((7, 3)), rng.standard_normal((5, 3)) + 5.0
    sa, sb = rng.standard_normal(7) + 1j * rng.standard_normal(7), rng.standard_normal(5) + 1j * rng.standard_normal(5)
    uab = oracle.field_direct(A, np.ones(7), k, sa, B)
    uba = oracle.field_direct(B, np.ones(5), k, sb, A)
    assert abs(np.dot(uab, sb) - np.dot(uba, sa)) < 1e-12 * abs(np.dot(uab, sb))
