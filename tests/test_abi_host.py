"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad input on the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1803_09948_gb300 as pkg
import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_09948_gb300 import build

    build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "hfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hfmm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert "hfmm_matvec" in names and "hfmm_solve" in names and len(names) >= 12
    lib = ctypes.CDLL(pkg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pkg.EXPORTED) == names


def test_default_config_and_status_strings():
    c = pkg.hfmm_default_config()
    assert c.leaf_max == 64 and c.restart == 30 and abs(c.tol - 1e-4) < 1e-18
    assert c.near_factor == 1.0 and c.p_min == 7
    assert c.m2l_tensor == 1 and c.adaptive == 0  # tensor-core M2L, uniform tree
    assert c.autotune == 0 and c.p2p_kernel == -1 and c.m2l_kernel == -1 and c.tc_group == 0 and c.overlap == -1
    for s in [0, 1, -1, -2, -3, -4, -5, -6]:
        assert pkg.hfmm_status_string(s) != "unknown status"
    assert pkg.hfmm_status_string(12345) == "unknown status"


def _create(V, F, k=1.0, k_im=0.0, **cfg):
    out = ctypes.c_void_p()
    st = pkg.hfmm_plan_create_raw(pkg.hfmm_default_config(**cfg), np.ascontiguousarray(V, dtype=np.float64),
                                  np.ascontiguousarray(F, dtype=np.int32), k, k_im, 0, out)
    return st, out


def test_invalid_arguments_are_rejected_on_the_host():
    V, F = synthetic.icosphere(0)
    assert _create(V, F, k=0.0)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, k=-1.0)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, k=float("nan"))[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, k=1.0, k_im=0.5)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, leaf_max=0)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, p_fixed=99)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, tol=0.0)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, quad_order=1)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, adaptive=2)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, m2l_tensor=-1)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, autotune=2)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, p2p_kernel=3)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, tc_group=12)[0] == pkg.HFMM_E_INVALID
    assert _create(V, F, overlap=3)[0] == pkg.HFMM_E_INVALID
    assert _create(V[:0], F)[0] == pkg.HFMM_E_INVALID          # no vertices
    assert _create(V, F[:0])[0] == pkg.HFMM_E_INVALID          # N = 0
    st, out = _create(V, F, k=0.0)
    assert not out.value  # nothing handed out on failure
    lib = pkg.lib()
    assert lib.hfmm_matvec(None, None, None, 1, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_matvec_host(None, None, None, 1, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_solve_group(None, 0, None, None, None, None, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_solve_group(None, 2, None, None, None, None, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_solver_info(None, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_solve(None, None, None, 1, None, None, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_num_points(None) == -1
    lib.hfmm_plan_destroy(None)  # no-op


def test_degenerate_meshes_are_rejected_on_the_host():
    V, F = synthetic.icosphere(0)
    Fz = F.copy()
    Fz[3] = [Fz[3][0], Fz[3][0], Fz[3][1]]  # repeated vertex: zero area
    st, _ = _create(V, Fz)
    assert st == pkg.HFMM_E_MESH and "zero-area" in pkg.hfmm_last_error()
    Vn = V.copy()
    Vn[5, 1] = np.nan
    assert _create(Vn, F)[0] == pkg.HFMM_E_MESH
    Fb = F.copy()
    Fb[0, 0] = V.shape[0]  # index out of range
    assert _create(V, Fb)[0] == pkg.HFMM_E_MESH
    Vc = V.copy()
    Vc[F[7]] = Vc[F[7][0]] + np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]])  # collinear
    assert _create(Vc, F)[0] == pkg.HFMM_E_MESH


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pkg.lib()


def test_package_does_not_reference_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_1803_09948_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "hfmm_oracle" not in txt, f


def test_tuner_rule_with_fake_timings():
    """The plan-time tuner keeps the fastest measured candidate, but keeps the default
    unless the fastest is at least 2 % faster; unmeasured entries (negative) are skipped."""
    P2P, M2L, GROUP, OVERLAP = 0, 1, 2, 3
    # near field: the default is the packed kernel (1)
    assert pkg.hfmm_tune_choose(P2P, [0.90, 1.00]) == 0           # staged 10 % faster
    assert pkg.hfmm_tune_choose(P2P, [0.99, 1.00]) == 1           # within noise: default kept
    assert pkg.hfmm_tune_choose(P2P, [1.20, 1.00]) == 1
    assert pkg.hfmm_tune_choose(P2P, [1.20, 1.00, 0.90]) == 2     # the pipelined kernel 10 % faster
    # M2L: the default is the source-stationary kernel (0)
    assert pkg.hfmm_tune_choose(M2L, [2.0, 0.5]) == 1
    assert pkg.hfmm_tune_choose(M2L, [1.0, 0.99]) == 0
    assert pkg.hfmm_tune_choose(GROUP, [1.2, 0.9, 1.0]) == 16     # default 32 at 1.0
    assert pkg.hfmm_tune_choose(GROUP, [0.99, 1.05, 1.0]) == 32   # 1 % faster only: default stays
    assert pkg.hfmm_tune_choose(GROUP, [-1.0, 0.7, -1.0]) == 16   # the only measured one
    assert pkg.hfmm_tune_choose(OVERLAP, [1.0, float("nan")]) == 0
    for bad in ([-1.0, -1.0], []):
        with pytest.raises(pkg.HfmmError):
            pkg.hfmm_tune_choose(P2P, bad)
    with pytest.raises(pkg.HfmmError):
        pkg.hfmm_tune_choose(7, [1.0, 2.0])
    with pytest.raises(pkg.HfmmError):
        pkg.hfmm_tune_choose(P2P, [1.0, 2.0, 3.0, 4.0])  # more values than candidates
