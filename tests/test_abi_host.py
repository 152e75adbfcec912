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
    assert _create(V[:0], F)[0] == pkg.HFMM_E_INVALID          # no vertices
    assert _create(V, F[:0])[0] == pkg.HFMM_E_INVALID          # N = 0
    st, out = _create(V, F, k=0.0)
    assert not out.value  # nothing handed out on failure
    lib = pkg.lib()
    assert lib.hfmm_matvec(None, None, None, 1, None) == pkg.HFMM_E_INVALID
    assert lib.hfmm_matvec_host(None, None, None, 1, None) == pkg.HFMM_E_INVALID
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
