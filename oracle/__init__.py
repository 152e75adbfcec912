"""Plain FP64 CPU oracle for the Helmholtz single-layer FMM matvec and solve.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg use it; the product library never
imports, loads or calls it, and it shares no code with the CUDA path.

Contents (paper: arXiv:1803.09948):
  * discrete operator Z (Sec. 2.2, Eq. 8-10 on flat triangles, 3 interior
    points each) by direct summation, as rows, as a dense matrix, and as the
    sparse near/self correction C = Z - Z_point;
  * FP64 FMM for the point part (Sec. 2.3, Eq. 11-14);
  * GMRES(m) with modified Gram-Schmidt and Givens rotations (the paper's
    solver, Sec. 5.1 / 6.4), dense LU for small systems;
  * the Mie series for the sound-soft sphere (analytic check of Sec. 6.4).
Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_points.argtypes = [_dp, _i32p, ctypes.c_int64, _dp, _dp, _i32p]
        L.or_mean_edge.argtypes = [_dp, _i32p, ctypes.c_int64]
        L.or_mean_edge.restype = ctypes.c_double
        L.or_tri_potential_1overR.argtypes = [_dp, _dp, _dp, _dp]
        L.or_tri_integrals.argtypes = [_dp, _dp, ctypes.c_double, _dp]
        L.or_correction_csr.argtypes = [_dp, _i32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        _i64p, _i64p, _dp]
        L.or_correction_csr.restype = ctypes.c_int64
        L.or_direct_rows.argtypes = [_dp, _i32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     _i64p, ctypes.c_int64, _dp, _dp, ctypes.c_int]
        L.or_direct_rows.restype = ctypes.c_int
        L.or_dense_Z.argtypes = [_dp, _i32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _dp]
        L.or_dense_Z.restype = ctypes.c_int
        L.or_near_sets.argtypes = [_dp, _i32p, ctypes.c_int64, ctypes.c_double, _i64p, _i32p]
        L.or_near_sets.restype = ctypes.c_int64
        L.or_point_sum.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_double, _dp, _dp]
        L.or_point_sum_rows.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_double, _i64p, ctypes.c_int64,
                                        _dp, _dp]
        L.or_fmm.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int, _ip]
        L.or_fmm.restype = ctypes.c_int
        L.or_sph_jn.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.or_sph_yn.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.or_ylm.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _mesh(V, F):
    return _f64(V), np.ascontiguousarray(F, dtype=np.int32)


# --------------------------------------------------------------------------
# discretisation
# --------------------------------------------------------------------------
def points(V, F):
    """Quadrature points X [N,3], weights W [N], triangle ids T [N]; N = 3 n_tri."""
    V, F = _mesh(V, F)
    nt = F.shape[0]
    X = np.empty((3 * nt, 3))
    W = np.empty(3 * nt)
    T = np.empty(3 * nt, dtype=np.int32)
    lib().or_points(_d(V), F.ctypes.data_as(_i32p), nt, _d(X), _d(W), T.ctypes.data_as(_i32p))
    return X, W, T


def mean_edge(V, F):
    V, F = _mesh(V, F)
    return lib().or_mean_edge(_d(V), F.ctypes.data_as(_i32p), F.shape[0])


def near_radius(V, F, near_factor):
    return near_factor * mean_edge(V, F)


class NearSetOverflow(RuntimeError):
    """A near set S(i) has more candidates than the oracle's fixed table holds."""


def near_sets(V, F, r_near):
    """S(i) for every point i: (ptr [N+1], idx) with idx[ptr[i]:ptr[i+1]] the sorted
    ids of the own triangle and of every triangle with a point within r_near of x_i."""
    V, F = _mesh(V, F)
    nt = F.shape[0]
    ptr = np.zeros(3 * nt + 1, dtype=np.int64)
    tot = lib().or_near_sets(_d(V), F.ctypes.data_as(_i32p), nt, float(r_near),
                             ptr.ctypes.data_as(_i64p), None)
    if tot < 0:
        raise NearSetOverflow("a near set exceeds the oracle's capacity; lower r_near")
    idx = np.empty(max(tot, 1), dtype=np.int32)
    lib().or_near_sets(_d(V), F.ctypes.data_as(_i32p), nt, float(r_near), ptr.ctypes.data_as(_i64p),
                       idx.ctypes.data_as(_i32p))
    return ptr, idx[:tot]


def tri_potential_1overR(x, v):
    x, v = _f64(x), _f64(v).reshape(9)
    I0 = np.zeros(1)
    I1 = np.zeros(3)
    lib().or_tri_potential_1overR(_d(x), _d(v), _d(I0), _d(I1))
    return I0[0], I1


def tri_integrals(x, v, k):
    """[int_T G(x,y) L_a(y) dS_y for a = 0,1,2], L_a = 2 lambda_a - 1/3."""
    x, v = _f64(x), _f64(v).reshape(9)
    out = np.zeros(6)
    lib().or_tri_integrals(_d(x), _d(v), float(k), _d(out))
    return out[0::2] + 1j * out[1::2]


def correction_csr(V, F, k, r_near):
    """C = Z - Z_point on the near/self sets, as a scipy CSR matrix (complex128)."""
    import scipy.sparse as sp

    V, F = _mesh(V, F)
    nt = F.shape[0]
    N = 3 * nt
    rowptr = np.zeros(N + 1, dtype=np.int64)
    nnz = lib().or_correction_csr(_d(V), F.ctypes.data_as(_i32p), nt, float(k), float(r_near),
                                  rowptr.ctypes.data_as(_i64p), None, None)
    if nnz < 0:
        raise NearSetOverflow("a near set exceeds the oracle's capacity; lower r_near")
    col = np.empty(max(nnz, 1), dtype=np.int64)
    val = np.empty(2 * max(nnz, 1))
    if lib().or_correction_csr(_d(V), F.ctypes.data_as(_i32p), nt, float(k), float(r_near),
                               rowptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p), _d(val)) < 0:
        raise NearSetOverflow("a near set exceeds the oracle's capacity; lower r_near")
    v = val[0:2 * nnz:2] + 1j * val[1:2 * nnz:2]
    return sp.csr_matrix((v, col[:nnz], rowptr), shape=(N, N))


def direct_rows(V, F, k, r_near, rows, sigma, mode=3):
    """Rows of Z sigma by direct summation (mode: 1 point part, 2 near/self part, 3 both)."""
    V, F = _mesh(V, F)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    s = _c128(sigma).view(np.float64)
    out = np.zeros(2 * rows.size)
    if lib().or_direct_rows(_d(V), F.ctypes.data_as(_i32p), F.shape[0], float(k), float(r_near),
                            rows.ctypes.data_as(_i64p), rows.size, _d(s), _d(out), int(mode)) < 0:
        raise NearSetOverflow("a near set exceeds the oracle's capacity; lower r_near")
    return out[0::2] + 1j * out[1::2]


def direct_matvec(V, F, k, r_near, sigma, mode=3):
    N = 3 * np.asarray(F).shape[0]
    return direct_rows(V, F, k, r_near, np.arange(N), sigma, mode)


def dense_Z(V, F, k, r_near):
    V, F = _mesh(V, F)
    N = 3 * F.shape[0]
    Z = np.zeros((N, N), dtype=np.complex128)
    if lib().or_dense_Z(_d(V), F.ctypes.data_as(_i32p), F.shape[0], float(k), float(r_near),
                        _d(Z.view(np.float64))) < 0:
        raise NearSetOverflow("a near set exceeds the oracle's capacity; lower r_near")
    return Z


def point_sum(X, W, k, sigma):
    """sum_{j != i} W_j G(x_i, x_j) sigma_j, no corrections."""
    X, W = _f64(X), _f64(W)
    s = _c128(sigma).view(np.float64)
    out = np.zeros(2 * W.size)
    lib().or_point_sum(_d(X), _d(W), W.size, float(k), _d(s), _d(out))
    return out[0::2] + 1j * out[1::2]


def point_sum_rows(X, W, k, sigma, rows):
    """Rows `rows` of point_sum (the same definition, O(N) per row)."""
    X, W = _f64(X), _f64(W)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    s = _c128(sigma).view(np.float64)
    out = np.zeros(2 * rows.size)
    lib().or_point_sum_rows(_d(X), _d(W), W.size, float(k), rows.ctypes.data_as(_i64p), rows.size, _d(s),
                            _d(out))
    return out[0::2] + 1j * out[1::2]


def fmm(X, W, k, sigma, depth=0, leaf_max=64, p_fixed=0, p_min=8, parts=3):
    """FP64 FMM of the point part; returns (values, info) with info = [L, p_1..p_L]."""
    X, W = _f64(X), _f64(W)
    s = _c128(sigma).view(np.float64)
    out = np.zeros(2 * W.size)
    info = np.zeros(24, dtype=np.int32)
    lib().or_fmm(_d(X), _d(W), W.size, float(k), int(depth), int(leaf_max), int(p_fixed), int(p_min),
                 _d(s), _d(out), int(parts), info.ctypes.data_as(_ip))
    L = int(info[0])
    return out[0::2] + 1j * out[1::2], [L] + [int(v) for v in info[1:L + 1]]


# --------------------------------------------------------------------------
# special functions (exported for their pins)
# --------------------------------------------------------------------------
def sph_jn(nmax, z):
    out = np.zeros(nmax + 1)
    lib().or_sph_jn(int(nmax), float(z), _d(out))
    return out


def sph_yn(nmax, z):
    out = np.zeros(nmax + 1)
    lib().or_sph_yn(int(nmax), float(z), _d(out))
    return out


def ylm(nmax, theta, phi):
    P = (nmax + 1) ** 2
    out = np.zeros(2 * P)
    lib().or_ylm(int(nmax), float(theta), float(phi), _d(out))
    return out[0::2] + 1j * out[1::2]


# --------------------------------------------------------------------------
# right-hand side, solver, analytic solution
# --------------------------------------------------------------------------
def plane_wave(X, k, d):
    """Incident field p_inc(x) = exp(i k d.x) at the points (Eq. 9's V_inc)."""
    d = np.asarray(d, dtype=np.float64)
    return np.exp(1j * k * (np.asarray(X) @ d))


def gmres(matvec, b, restart=30, tol=1e-4, maxiter=1000, x0=None):
    """Restarted GMRES(m) (Saad & Schultz), modified Gram-Schmidt, Givens rotations.

    Stops when the recurrence residual |g_{j+1}| / ||b|| <= tol; the true
    residual is recomputed at every restart and at exit.
    Returns (x, iterations, true relative residual, history of recurrence residuals).
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, []
    hist = []
    it = 0
    r = b - matvec(x) if x0 is not None else b.copy()
    beta = np.linalg.norm(r)
    while it < maxiter:
        if beta / bnorm <= tol:
            break
        m = restart
        Vb = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        j_done = 0
        for j in range(m):
            w = matvec(Vb[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                Vb[j + 1] = w / H[j + 1, j]
            # rotation i acts on rows (i, i+1) as [[conj(c), conj(s)], [-s, c]]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a / den
                sn[j] = bb / den
            H[j, j] = np.conj(cs[j]) * a + np.conj(sn[j]) * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Vb[:j_done].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if hist and hist[-1] <= tol:
            break
    return x, it, float(np.linalg.norm(b - matvec(x)) / bnorm), hist


def dense_solve(Z, b):
    return np.linalg.solve(Z, b)


def mie_surface_q(X, k, a=1.0, d=(0.0, 0.0, 1.0), nmax=None):
    """Exact surface Neumann data of the sound-soft sphere of radius a hit by
    exp(i k d.x):  q(theta) = -(i/(k a^2)) sum_n i^n (2n+1) P_n(cos theta) / h_n(ka),
    evaluated at the radial projection of each point onto the sphere."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn

    X = np.asarray(X, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    ct = (X @ d) / np.linalg.norm(X, axis=1)
    ka = k * a
    if nmax is None:
        nmax = int(ka + 10 * max(1.0, ka) ** (1.0 / 3.0) + 10)
    q = np.zeros(X.shape[0], dtype=np.complex128)
    for n in range(nmax + 1):
        hn = spherical_jn(n, ka) + 1j * spherical_yn(n, ka)
        q += (1j ** n) * (2 * n + 1) * eval_legendre(n, ct) / hn
    return -(1j / (k * a * a)) * q


def field_direct(X, W, k, sigma, targets):
    """Off-surface single-layer potential by its definition (point rule of Eq. 10 with
    the targets apart from the points):  u(t) = sum_j W_j exp(i k |t - x_j|) / (4 pi |t - x_j|) sigma_j."""
    X, W, T = _f64(X).reshape(-1, 3), _f64(W), _f64(targets).reshape(-1, 3)
    s = _c128(sigma) * W
    out = np.zeros(T.shape[0], dtype=np.complex128)
    for a in range(0, T.shape[0], 64):
        R = np.linalg.norm(T[a:a + 64, None, :] - X[None, :, :], axis=2)
        out[a:a + 64] = (np.exp(1j * k * R) / (4.0 * np.pi * R)) @ s
    return out


def mie_scattered(T, k, a=1.0, d=(0.0, 0.0, 1.0), nmax=None):
    """Exact scattered field outside the sound-soft sphere of radius a hit by exp(i k d.x):
    p_s(r, theta) = -sum_n i^n (2n+1) j_n(ka) / h_n(ka) h_n(kr) P_n(cos theta)  (h = h^(1))."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn

    T = np.asarray(T, dtype=np.float64).reshape(-1, 3)
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    r = np.linalg.norm(T, axis=1)
    ct = (T @ d) / r
    ka = k * a
    if nmax is None:
        nmax = int(ka + 10 * max(1.0, ka) ** (1.0 / 3.0) + 10)
    p = np.zeros(T.shape[0], dtype=np.complex128)
    for n in range(nmax + 1):
        ha = spherical_jn(n, ka) + 1j * spherical_yn(n, ka)
        hr = spherical_jn(n, k * r) + 1j * spherical_yn(n, k * r)
        p -= (1j ** n) * (2 * n + 1) * spherical_jn(n, ka) / ha * hr * eval_legendre(n, ct)
    return p
