"""Every selectable kernel variant against the FP64 oracle.

The configuration can pin (or leave to the plan-time tuner) the near-field kernel
(p2p_kernel 0: four lanes per target; 1: packed FP32x2 pairs of sources; 2: the packed
arithmetic in persistent blocks with the next leaf's sources loaded by cp.async), the matvec
form (overlap 0: stages one after another; 1: near field and correction on a second
branch beside the far field, captured once as a CUDA graph) and the tensor-core group
size.  Whatever the tuner picks must meet the same bars as the defaults:
  near field vs the oracle's near field on the same tree   1e-5
  matvec vs the oracle's direct sum                        1e-4
  the two matvec forms against each other                  1e-6 (summation order only)
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _apply(plan, s, parts=7):
    d = torch.from_numpy(np.ascontiguousarray(s).astype(np.complex64)).cuda()
    o = torch.empty_like(d)
    if parts == 7:
        plan.matvec(d, o)
    else:
        plan.matvec_parts(d, o, parts)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def c1():
    V, F = synthetic.sphere_mesh(3)
    s = synthetic.random_density(3 * F.shape[0], seed=0)
    r = oracle.near_radius(V, F, 1.0)
    X, W, _ = oracle.points(V, F)
    near, _ = oracle.fmm(X, W, 1.0, s, leaf_max=64, p_fixed=8, parts=1)
    return dict(V=V, F=F, s=s, ref=oracle.direct_matvec(V, F, 1.0, r, s), near=near)


@pytest.mark.parametrize("p2p", [0, 1, 2])
@pytest.mark.parametrize("overlap", [0, 1])
def test_matvec_variants_against_oracle(c1, p2p, overlap):
    plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=8, leaf_max=64, p2p_kernel=p2p, overlap=overlap)
    try:
        assert rel(_apply(plan, c1["s"], parts=1), c1["near"]) < 1e-5
        got = _apply(plan, c1["s"])
        assert rel(got, c1["ref"]) < 1e-4
        again = _apply(plan, c1["s"])  # a replay of the captured graph
        assert rel(again, got) < 1e-6
        assert plan.device_status() == pkg.HFMM_OK
    finally:
        plan.close()


def test_overlapped_and_sequential_forms_agree(c1):
    a = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=8, overlap=0)
    b = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=8, overlap=1)
    try:
        assert rel(_apply(b, c1["s"]), _apply(a, c1["s"])) < 1e-6
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("p2p", [0, 1, 2])
def test_near_field_kernels_all_pairs_and_polynomial_edge(p2p):
    """One leaf holding every point (targets loop over several rounds of 128 threads),
    and the polynomial's top range on the corner-lattice soup."""
    V, F = synthetic.sphere_mesh(2)
    plan = pkg.Plan(V, F, 3.0, leaf_max=10 ** 6, p2p_kernel=p2p)
    try:
        X, W, _ = oracle.points(V, F)
        s = synthetic.random_density(plan.n, seed=3)
        assert rel(_apply(plan, s, parts=1), oracle.point_sum(X, W, 3.0, s)) < 1e-5
    finally:
        plan.close()
    V, F = synthetic.corner_lattice_soup(8, 0.03, seed=1, size=2e-3)
    k = 1.824
    plan = pkg.Plan(V, F, k, leaf_max=64, p_fixed=4, p2p_kernel=p2p)
    try:
        X, W, _ = oracle.points(V, F)
        s = synthetic.random_density(plan.n, seed=8)
        near, info = oracle.fmm(X, W, k, s, leaf_max=64, p_fixed=4, parts=1)
        assert info[0] == plan.info()["depth"]
        assert rel(_apply(plan, s, parts=1), near) < 1e-5
    finally:
        plan.close()


@pytest.mark.parametrize("p2p", [0, 1, 2])
@pytest.mark.parametrize("level,leaf", [(0, 4), (1, 16), (2, 20)])
def test_near_field_kernels_small_and_ragged(p2p, level, leaf):
    """Leaves of 1..20 points: odd self segments, padding pairs, one thread group per target."""
    V, F = synthetic.icosphere(level)
    k = 2.5
    plan = pkg.Plan(V, F, k, p_fixed=10, leaf_max=leaf, p2p_kernel=p2p, overlap=1)
    try:
        s = synthetic.random_density(plan.n, seed=level)
        ref = oracle.direct_matvec(V, F, k, oracle.near_radius(V, F, 1.0), s)
        assert rel(_apply(plan, s), ref) < 1e-4
    finally:
        plan.close()


@pytest.mark.parametrize("p", [3, 4, 5, 6, 7])
def test_target_stationary_m2l_against_simt_and_oracle(c1, p):
    """Target-stationary tensor-core M2L (canonical operators of the offsets' reflection
    classes, signed permutations of the gathered multipoles and of the product's rows) against
    the FP32 SIMT far field of the same plan and the oracle's direct sum; p = 4, 6 give odd
    (p+1)^2 (25, 49): the real form's imaginary block then starts at an even K offset."""
    ts = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=p, m2l_kernel=1)
    simt = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=p, m2l_tensor=0)
    try:
        assert ts.tuning()["m2l_kernel"]["choice"] == 1
        far_ts = _apply(ts, c1["s"], parts=2)
        far_simt = _apply(simt, c1["s"], parts=2)
        assert ts.device_status() == pkg.HFMM_OK
        assert np.linalg.norm(far_ts - far_simt) < 3e-5 * np.linalg.norm(far_simt)
        e_ts, e_simt = rel(_apply(ts, c1["s"]), c1["ref"]), rel(_apply(simt, c1["s"]), c1["ref"])
        assert e_ts < e_simt + 2e-6
        if p == 7:
            assert e_ts < 1e-4
    finally:
        ts.close()
        simt.close()


def test_target_stationary_m2l_full_size_far_field():
    """491,520-point sphere at k = 10 (levels 3-6 at p = 7 on the tensor cores; 1.1 M
    translations in 18k-box levels, many tiles): far field against the SIMT form."""
    V, F = synthetic.workload_mesh("sphere_163840")
    ts = pkg.Plan(V, F, 10.0, m2l_kernel=1)
    simt = pkg.Plan(V, F, 10.0, m2l_tensor=0)
    try:
        s = synthetic.random_density(ts.n, seed=4)
        far_ts = _apply(ts, s, parts=2)
        far_simt = _apply(simt, s, parts=2)
        assert ts.device_status() == pkg.HFMM_OK
        assert rel(far_ts, far_simt) < 3e-5
    finally:
        ts.close()
        simt.close()


@pytest.mark.parametrize("group", [8, 16])
def test_tensor_core_group_sizes(c1, group):
    plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=7, tc_group=group)
    try:
        assert rel(_apply(plan, c1["s"]), c1["ref"]) < 1e-4
        assert plan.device_status() == pkg.HFMM_OK
    finally:
        plan.close()


def test_solve_through_the_captured_graph(c1):
    """GMRES calls the matvec through the captured two-branch graph."""
    plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=8, overlap=1, p2p_kernel=1)
    try:
        b = torch.empty(plan.n, dtype=torch.complex64, device="cuda")
        plan.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, its, rr = plan.solve(b, x)
        assert st == pkg.HFMM_OK and rr[0] <= 1e-4
        X, _, _ = oracle.points(c1["V"], c1["F"])
        Z = oracle.dense_Z(c1["V"], c1["F"], 1.0, oracle.near_radius(c1["V"], c1["F"], 1.0))
        bb = oracle.plane_wave(X, 1.0, (0, 0, 1))
        xg = x.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(Z @ xg - bb) / np.linalg.norm(bb) < 2e-4
    finally:
        plan.close()


def test_autotuned_plan_meets_the_bars(c1):
    """autotune = 1: every open choice is timed at plan creation; the plan reports a valid
    choice and the timings of the candidates it compared, and its matvec meets the bar."""
    plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=7, autotune=1)
    try:
        t = plan.tuning()
        for name, cands in pkg.TUNABLES:
            assert t[name]["choice"] in cands
        assert set(t["p2p_kernel"]["ms"]) == {0, 1, 2} and set(t["overlap"]["ms"]) == {0, 1}
        assert set(t["m2l_kernel"]["ms"]) == {0, 1}
        assert all(v > 0 for q in t.values() for v in q["ms"].values())
        assert rel(_apply(plan, c1["s"]), c1["ref"]) < 1e-4
        assert plan.device_status() == pkg.HFMM_OK
    finally:
        plan.close()
