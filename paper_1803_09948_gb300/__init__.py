"""Python binding of the GB300 Helmholtz FMM library (libhfmm.so, C ABI in include/hfmm.h).

Argument marshalling only: every step of the matvec and the solve runs in the
library's CUDA kernels.  Device vectors are torch complex64 CUDA tensors (or
raw device pointers); PyTorch provides device memory and streams.  There is no
CPU fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfmm.so")
_lib = None

HFMM_OK = 0
HFMM_NOT_CONVERGED = 1
HFMM_E_INVALID = -1
HFMM_E_MESH = -2
HFMM_E_NOMEM = -3
HFMM_E_CUDA = -4
HFMM_E_TIMEOUT = -5
HFMM_E_OVERFLOW = -6

EXPORTED = [
    "hfmm_default_config", "hfmm_plan_create", "hfmm_plan_destroy", "hfmm_num_points", "hfmm_points",
    "hfmm_plan_info", "hfmm_matvec", "hfmm_matvec_parts", "hfmm_direct", "hfmm_rhs_planewave",
    "hfmm_solve", "hfmm_solve_refined", "hfmm_status_string", "hfmm_last_error", "hfmm_matvec_timed",
    "hfmm_launch_count", "hfmm_plan_costs", "hfmm_point_sum_noalloc", "hfmm_device_status", "hfmm_field",
    "hfmm_matvec_host", "hfmm_plan_tuning", "hfmm_tune_choose", "hfmm_matvec_df", "hfmm_solver_info",
    "hfmm_solve_group",
]
HFMM_NOALLOC_MAX_POINTS = 262144
STAGES = ["prep", "p2p", "p2m", "m2m", "m2l_simt", "m2l", "l2l", "l2p", "corr", "output"]


class hfmm_config(ctypes.Structure):
    _fields_ = [
        ("leaf_max", ctypes.c_int),
        ("depth", ctypes.c_int),
        ("p_fixed", ctypes.c_int),
        ("p_min", ctypes.c_int),
        ("near_factor", ctypes.c_double),
        ("quad_order", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("mem_budget_bytes", ctypes.c_double),
        ("m2l_tensor", ctypes.c_int),
        ("adaptive", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("p2p_kernel", ctypes.c_int),
        ("m2l_kernel", ctypes.c_int),
        ("tc_group", ctypes.c_int),
        ("overlap", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


class HfmmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = hfmm_last_error() if _lib is not None else ""
        super().__init__(f"{where}: {hfmm_status_string(status)} ({status}) {detail}".strip())


def lib():
    """Loads libhfmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.hfmm_default_config.argtypes = [ctypes.POINTER(hfmm_config)]
        L.hfmm_default_config.restype = None
        L.hfmm_plan_create.argtypes = [ctypes.POINTER(hfmm_config), dp, i64, ctypes.POINTER(ctypes.c_int32), i64,
                                       ctypes.c_double, ctypes.c_double, vp, ctypes.POINTER(vp)]
        L.hfmm_plan_destroy.argtypes = [vp]
        L.hfmm_plan_destroy.restype = None
        L.hfmm_num_points.argtypes = [vp]
        L.hfmm_num_points.restype = i64
        L.hfmm_points.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int32)]
        L.hfmm_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(i64)]
        L.hfmm_matvec.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.hfmm_matvec_parts.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.hfmm_matvec_host.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.hfmm_matvec_df.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.hfmm_solver_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.hfmm_solve_group.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(ctypes.c_int), dp, vp]
        L.hfmm_plan_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        L.hfmm_tune_choose.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
        L.hfmm_direct.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.hfmm_rhs_planewave.argtypes = [vp, dp, ctypes.c_int, vp, vp]
        L.hfmm_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, vp]
        L.hfmm_field.argtypes = [vp, vp, dp, i64, vp, vp]
        L.hfmm_solve_refined.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), dp, vp]
        L.hfmm_status_string.argtypes = [ctypes.c_int]
        L.hfmm_status_string.restype = ctypes.c_char_p
        L.hfmm_matvec_timed.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_float), vp]
        L.hfmm_plan_costs.argtypes = [vp, dp]
        L.hfmm_device_status.argtypes = [vp, vp]
        L.hfmm_point_sum_noalloc.argtypes = [vp, vp, i64, ctypes.c_double, vp, vp, vp]
        L.hfmm_launch_count.argtypes = [vp]
        L.hfmm_launch_count.restype = i64
        L.hfmm_last_error.argtypes = []
        L.hfmm_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status, where):
    if status < 0:
        raise HfmmError(status, where)
    return status


def _ptr(x):
    """Device (or host) address of a torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _vec(t, n, nrhs, name):
    import torch

    if isinstance(t, int):
        return
    if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous() and t.numel() == n * nrhs):
        raise ValueError(f"{name}: expected a contiguous complex64 CUDA tensor of {n * nrhs} elements")


# ---------------------------------------------------------------- ABI mirrors
def hfmm_default_config(**overrides):
    c = hfmm_config()
    lib().hfmm_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def hfmm_status_string(status):
    return lib().hfmm_status_string(int(status)).decode()


def hfmm_last_error():
    return lib().hfmm_last_error().decode()


def hfmm_plan_create(cfg, vertices, tris, k_re, k_im=0.0, stream=None):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    out = ctypes.c_void_p()
    st = hfmm_plan_create_raw(cfg, V, F, k_re, k_im, stream, out)
    _check(st, "hfmm_plan_create")
    return out


def hfmm_plan_create_raw(cfg, V, F, k_re, k_im, stream, out):
    return lib().hfmm_plan_create(
        ctypes.byref(cfg), V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), V.shape[0] if V.ndim else 0,
        F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), F.shape[0] if F.ndim else 0, float(k_re), float(k_im),
        _stream(stream), ctypes.byref(out))


def hfmm_plan_destroy(plan):
    lib().hfmm_plan_destroy(plan)


def hfmm_num_points(plan):
    return int(lib().hfmm_num_points(plan))


def hfmm_points(plan):
    n = hfmm_num_points(plan)
    xyz = np.empty((n, 3))
    w = np.empty(n)
    tri = np.empty(n, dtype=np.int32)
    _check(lib().hfmm_points(plan, xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "hfmm_points")
    return xyz, w, tri


def hfmm_plan_info(plan):
    depth = ctypes.c_int()
    orders = (ctypes.c_int * 32)()
    nl, nnz, m2l, by = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().hfmm_plan_info(plan, ctypes.byref(depth), orders, ctypes.byref(nl), ctypes.byref(nnz),
                                ctypes.byref(m2l), ctypes.byref(by)), "hfmm_plan_info")
    return {"depth": depth.value, "orders": [orders[l] for l in range(depth.value + 1)], "n_leaves": nl.value,
            "corr_nnz": nnz.value, "m2l_translations": m2l.value, "device_bytes": by.value}


def hfmm_matvec(plan, density, potential, nrhs=1, stream=None):
    n = hfmm_num_points(plan)
    _vec(density, n, nrhs, "density")
    _vec(potential, n, nrhs, "potential")
    _check(lib().hfmm_matvec(plan, _ptr(density), _ptr(potential), int(nrhs), _stream(stream)), "hfmm_matvec")


def hfmm_matvec_host(plan, density, potential, nrhs=1, stream=None):
    """density / potential: contiguous complex64 CPU tensors (page-locked for speed) of N x nrhs."""
    import torch

    n = hfmm_num_points(plan)
    for t, name in ((density, "density"), (potential, "potential")):
        if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == torch.complex64
                and t.is_contiguous() and t.numel() == n * nrhs):
            raise ValueError(f"{name}: expected a contiguous complex64 CPU tensor of {n * nrhs} elements")
    _check(lib().hfmm_matvec_host(plan, _ptr(density), _ptr(potential), int(nrhs), _stream(stream)),
           "hfmm_matvec_host")


def _df_vec(t, n, name):
    import torch

    if isinstance(t, int):
        return
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == 4 * n):
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor of N x 4 (re_hi, im_hi, re_lo, im_lo)")


def df_from_complex(x, device="cuda"):
    """complex128 numpy vector -> N x 4 float32 tensor (re_hi, im_hi, re_lo, im_lo), hi + lo = x."""
    import numpy as np
    import torch

    x = np.asarray(x, dtype=np.complex128)
    hi = x.astype(np.complex64)
    lo = (x - hi.astype(np.complex128)).astype(np.complex64)
    out = np.stack([hi.real, hi.imag, lo.real, lo.imag], axis=1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(out)).to(device)


def df_to_complex(t):
    """N x 4 float32 tensor (re_hi, im_hi, re_lo, im_lo) -> complex128 numpy vector hi + lo."""
    import numpy as np

    a = t.detach().cpu().numpy().astype(np.float64).reshape(-1, 4)
    return (a[:, 0] + a[:, 2]) + 1j * (a[:, 1] + a[:, 3])


def hfmm_matvec_df(plan, density_df, potential_df, parts=7, stream=None):
    """Double-float matvec (precision = 1 plans): N x 4 float32 CUDA tensors in and out."""
    n = hfmm_num_points(plan)
    _df_vec(density_df, n, "density_df")
    _df_vec(potential_df, n, "potential_df")
    _check(lib().hfmm_matvec_df(plan, _ptr(density_df), _ptr(potential_df), int(parts), _stream(stream)),
           "hfmm_matvec_df")


def hfmm_matvec_parts(plan, density, potential, parts, nrhs=1, stream=None):
    n = hfmm_num_points(plan)
    _vec(density, n, nrhs, "density")
    _vec(potential, n, nrhs, "potential")
    _check(lib().hfmm_matvec_parts(plan, _ptr(density), _ptr(potential), int(nrhs), int(parts), _stream(stream)),
           "hfmm_matvec_parts")


def hfmm_matvec_timed(plan, density, potential, stream=None):
    """One matvec with per-stage device times (ms), keyed by STAGES."""
    n = hfmm_num_points(plan)
    _vec(density, n, 1, "density")
    _vec(potential, n, 1, "potential")
    ms = (ctypes.c_float * len(STAGES))()
    _check(lib().hfmm_matvec_timed(plan, _ptr(density), _ptr(potential), ms, _stream(stream)), "hfmm_matvec_timed")
    return dict(zip(STAGES, [float(v) for v in ms]))


def hfmm_plan_costs(plan):
    keys = ["p2p_pairs", "m2l_cmacs", "m2m_l2l_cmacs", "corr_nnz", "n_points", "coefficients", "m2l_tc_cmacs",
            "m2l_tc_translations", "leaf_coefficients", "level2_coefficients", "multipole_coefficients",
            "levelL_coefficients"]
    c = (ctypes.c_double * len(keys))()
    _check(lib().hfmm_plan_costs(plan, c), "hfmm_plan_costs")
    return dict(zip(keys, [float(v) for v in c]))


TUNABLES = [("p2p_kernel", [0, 1, 2]), ("m2l_kernel", [0, 1]), ("tc_group", [8, 16, 32]), ("overlap", [0, 1])]


def hfmm_plan_tuning(plan):
    """{tunable: {"choice": value, "ms": {candidate: device ms of one matvec}}} (timed ones only)."""
    ch = (ctypes.c_int * 4)()
    ms = (ctypes.c_float * 16)()
    _check(lib().hfmm_plan_tuning(plan, ch, ms), "hfmm_plan_tuning")
    out = {}
    for a, (name, cands) in enumerate(TUNABLES):
        timed = {c: float(ms[4 * a + q]) for q, c in enumerate(cands) if ms[4 * a + q] >= 0}
        out[name] = {"choice": int(ch[a]), "ms": timed}
    return out


def hfmm_tune_choose(tunable, ms):
    """The tuner's rule on given timings (ms per candidate, negative = not measured)."""
    arr = (ctypes.c_float * len(ms))(*[float(v) for v in ms])
    v = ctypes.c_int()
    _check(lib().hfmm_tune_choose(int(tunable), arr, len(ms), ctypes.byref(v)), "hfmm_tune_choose")
    return int(v.value)


def hfmm_point_sum_noalloc(xyz, w, density, potential, k, stream=None):
    """Point sum through the scratch-free entry point; xyz [n,3] and w [n] are
    float64 CUDA tensors, density / potential complex64 CUDA tensors."""
    import torch

    n = int(w.numel())
    if not (xyz.is_cuda and w.is_cuda and xyz.dtype == torch.float64 and w.dtype == torch.float64
            and xyz.is_contiguous() and w.is_contiguous() and xyz.numel() == 3 * n):
        raise ValueError("xyz / w: expected contiguous float64 CUDA tensors of 3n and n elements")
    _vec(density, n, 1, "density")
    _vec(potential, n, 1, "potential")
    return _check(lib().hfmm_point_sum_noalloc(_ptr(xyz), _ptr(w), n, float(k), _ptr(density), _ptr(potential),
                                               _stream(stream)), "hfmm_point_sum_noalloc")


def hfmm_device_status(plan, stream=None):
    """HFMM_OK, or HFMM_E_TIMEOUT if a kernel's bounded wait gave up since the last call."""
    return int(lib().hfmm_device_status(plan, _stream(stream)))


def hfmm_launch_count(plan):
    return int(lib().hfmm_launch_count(plan))


def hfmm_direct(plan, density, potential, nrhs=1, stream=None):
    n = hfmm_num_points(plan)
    _vec(density, n, nrhs, "density")
    _vec(potential, n, nrhs, "potential")
    _check(lib().hfmm_direct(plan, _ptr(density), _ptr(potential), int(nrhs), _stream(stream)), "hfmm_direct")


def hfmm_rhs_planewave(plan, dirs, rhs_out, stream=None):
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    n = hfmm_num_points(plan)
    _vec(rhs_out, n, d.shape[0], "rhs_out")
    _check(lib().hfmm_rhs_planewave(plan, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), d.shape[0],
                                    _ptr(rhs_out), _stream(stream)), "hfmm_rhs_planewave")


def hfmm_solve(plan, rhs, x_out, nrhs=1, stream=None):
    """Returns (status, iterations[nrhs], relative residuals[nrhs])."""
    n = hfmm_num_points(plan)
    _vec(rhs, n, nrhs, "rhs")
    _vec(x_out, n, nrhs, "x_out")
    its = (ctypes.c_int * nrhs)()
    rr = (ctypes.c_double * nrhs)()
    st = _check(lib().hfmm_solve(plan, _ptr(rhs), _ptr(x_out), int(nrhs), its, rr, _stream(stream)), "hfmm_solve")
    return st, list(its), list(rr)


def hfmm_field(plan, density, targets, field_out, stream=None):
    """Single-layer potential of `density` at off-surface `targets` (host array [n][3])."""
    n = hfmm_num_points(plan)
    _vec(density, n, 1, "density")
    T = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, 3))
    _vec(field_out, T.shape[0], 1, "field_out")
    _check(lib().hfmm_field(plan, _ptr(density), T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), T.shape[0],
                            _ptr(field_out), _stream(stream)), "hfmm_field")


def hfmm_solve_group(plans, rhs, x_out, stream=None):
    """G single right-hand-side solves on distinct plans, each restart cycle of all of them in one
    shared graph launch.  plans: Plan objects or handles; rhs / x_out: complex64 CUDA tensors of
    each plan's N.  Returns (status, iterations[G], true relative residuals[G])."""
    hs = [p.handle if isinstance(p, Plan) else p for p in plans]
    G = len(hs)
    if not (len(rhs) == len(x_out) == G):
        raise ValueError("plans, rhs and x_out must have the same length")
    for h, b, x in zip(hs, rhs, x_out):
        n = hfmm_num_points(h)
        _vec(b, n, 1, "rhs")
        _vec(x, n, 1, "x_out")
    vp = ctypes.c_void_p
    pa = (vp * G)(*[h.value if isinstance(h, vp) else h for h in hs])
    ra = (vp * G)(*[b.data_ptr() for b in rhs])
    xa = (vp * G)(*[x.data_ptr() for x in x_out])
    its = (ctypes.c_int * G)()
    rr = (ctypes.c_double * G)()
    st = _check(lib().hfmm_solve_group(pa, G, ra, xa, its, rr, _stream(stream)), "hfmm_solve_group")
    return st, list(its), list(rr)


def hfmm_solve_refined(inner, outer, rhs, x_out, tol=1e-6, max_outer=10, stream=None):
    """Mixed-precision refinement: GMRES on `inner`, residuals with `outer` in double-float.
    Returns (status, refinement steps, inner GMRES iterations, final relative residual)."""
    n = hfmm_num_points(inner)
    _vec(rhs, n, 1, "rhs")
    _vec(x_out, n, 1, "x_out")
    oi, ii, rr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = _check(lib().hfmm_solve_refined(inner, outer, _ptr(rhs), _ptr(x_out), float(tol), int(max_outer),
                                         ctypes.byref(oi), ctypes.byref(ii), ctypes.byref(rr), _stream(stream)),
                "hfmm_solve_refined")
    return st, oi.value, ii.value, rr.value


class Plan:
    """Owning wrapper: Plan(vertices, tris, k, **config) ... plan.close()."""

    def __init__(self, vertices, tris, k, stream=None, **cfg):
        self.cfg = hfmm_default_config(**cfg)
        self.handle = hfmm_plan_create(self.cfg, vertices, tris, k, 0.0, stream)
        self.n = hfmm_num_points(self.handle)
        self.k = float(k)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            hfmm_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return hfmm_plan_info(self.handle)

    def points(self):
        return hfmm_points(self.handle)

    def matvec(self, density, potential, nrhs=1, stream=None):
        hfmm_matvec(self.handle, density, potential, nrhs, stream)

    def matvec_host(self, density, potential, nrhs=1, stream=None):
        hfmm_matvec_host(self.handle, density, potential, nrhs, stream)

    def solver_info(self):
        """{'cycle_graph': 1 if the last single-RHS solve ran its GMRES cycles as graph launches}."""
        v = ctypes.c_int()
        _check(lib().hfmm_solver_info(self.handle, ctypes.byref(v)), "hfmm_solver_info")
        return {"cycle_graph": v.value}

    def matvec_df(self, density_df, potential_df, parts=7, stream=None):
        hfmm_matvec_df(self.handle, density_df, potential_df, parts, stream)

    def matvec_parts(self, density, potential, parts, nrhs=1, stream=None):
        hfmm_matvec_parts(self.handle, density, potential, parts, nrhs, stream)

    def matvec_timed(self, density, potential, stream=None):
        return hfmm_matvec_timed(self.handle, density, potential, stream)

    def costs(self):
        return hfmm_plan_costs(self.handle)

    def tuning(self):
        return hfmm_plan_tuning(self.handle)

    def device_status(self, stream=None):
        return hfmm_device_status(self.handle, stream)

    def launch_count(self):
        return hfmm_launch_count(self.handle)

    def direct(self, density, potential, nrhs=1, stream=None):
        hfmm_direct(self.handle, density, potential, nrhs, stream)

    def rhs_planewave(self, dirs, rhs_out, stream=None):
        hfmm_rhs_planewave(self.handle, dirs, rhs_out, stream)

    def solve(self, rhs, x_out, nrhs=1, stream=None):
        return hfmm_solve(self.handle, rhs, x_out, nrhs, stream)

    def field(self, density, targets, field_out, stream=None):
        hfmm_field(self.handle, density, targets, field_out, stream)

    def solve_refined(self, outer, rhs, x_out, tol=1e-6, max_outer=10, stream=None):
        """GMRES on this plan inside a refinement loop whose residuals use `outer`."""
        return hfmm_solve_refined(self.handle, outer.handle, rhs, x_out, tol, max_outer, stream)
