"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative 2-norm over the whole output vector):
  near field (P2P) and direct summation   1e-5   (FP32 arithmetic, FP64 oracle)
  sparse self/near correction             1e-5
  FMM matvec vs direct summation          1e-4   (expansion order p = 8 on the small sphere)
  GMRES solution                          see the individual tests
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1803_09948_gb300 as pkg
import synthetic

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).astype(np.complex64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _apply(plan, s, parts=7, nrhs=1):
    d = _dev(s.reshape(-1))
    o = torch.empty_like(d)
    if parts == 7:
        plan.matvec(d, o, nrhs)
    else:
        plan.matvec_parts(d, o, parts, nrhs)
    return _host(o).reshape(s.shape)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def c1():
    """Small configuration: unit sphere, 1,280 triangles (N = 3,840), k = 1, p = 8, leaf <= 64."""
    V, F = synthetic.sphere_mesh(3)
    plan = pkg.Plan(V, F, 1.0, p_fixed=8, leaf_max=64)
    s = synthetic.random_density(plan.n, seed=0)
    r = oracle.near_radius(V, F, plan.cfg.near_factor)
    ref = oracle.direct_matvec(V, F, 1.0, r, s)
    yield dict(V=V, F=F, plan=plan, s=s, r=r, ref=ref, k=1.0)
    plan.close()


def test_points_match_oracle(c1):
    X, W, T = c1["plan"].points()
    Xo, Wo, To = oracle.points(c1["V"], c1["F"])
    assert np.array_equal(T, To)
    assert np.max(np.abs(X - Xo)) <= 1e-15 and np.max(np.abs(W - Wo)) <= 1e-17


def test_plan_shape_c1(c1):
    info = c1["plan"].info()
    assert info["depth"] == 3 and info["orders"][2:] == [8, 8]
    assert info["m2l_translations"] > 0 and info["corr_nnz"] >= 3 * c1["plan"].n


def test_p2p_all_pairs_against_oracle():
    """One leaf holding every point: the near field is the whole point sum."""
    V, F = synthetic.sphere_mesh(2)
    plan = pkg.Plan(V, F, 3.0, leaf_max=10 ** 6)
    try:
        assert plan.info()["depth"] == 0
        X, W, _ = oracle.points(V, F)
        s = synthetic.random_density(plan.n, seed=3)
        got = _apply(plan, s, parts=1)
        assert rel(got, oracle.point_sum(X, W, 3.0, s)) < 1e-5
    finally:
        plan.close()


def test_p2p_neighbour_leaves_against_oracle(c1):
    """Leaf tiles and neighbour lists (polynomial kernel path, kR <= 0.87)."""
    X, W, _ = oracle.points(c1["V"], c1["F"])
    near, info = oracle.fmm(X, W, 1.0, c1["s"], leaf_max=64, p_fixed=8, parts=1)
    assert info[0] == 3
    assert rel(_apply(c1["plan"], c1["s"], parts=1), near) < 1e-5


def test_p2p_top_of_polynomial_range_against_oracle():
    """The polynomial kernel (cos and sinc fitted in u = (kR)^2 on [0, 2.5]) at the top
    of its range.  Small triangles sit near the corners of every leaf of a depth-3 tree,
    so neighbour pairs reach u ~ 2.39 (the plan admits the polynomial up to
    12 (k side)^2 <= 2.5); compared with the oracle's near field on the same tree.
    Triangle size (2e-3) against leaf side (0.25) keeps float32 leaf-local positions'
    rounding, emulated on the CPU, at 2.2e-6 of the result (with 3e-4 triangles it alone
    is 1.45e-5: the same-triangle pairs dominate and their distance loses digits)."""
    V, F = synthetic.corner_lattice_soup(8, 0.03, seed=1, size=2e-3)
    k = 1.824
    plan = pkg.Plan(V, F, k, leaf_max=64, p_fixed=4)
    try:
        L = plan.info()["depth"]
        assert L == 3
        X, W, _ = oracle.points(V, F)
        lo, hi = X.min(0), X.max(0)
        side = 2.0 ** np.ceil(np.log2((hi - lo).max())) / 2 ** L
        assert 12.0 * (k * side) ** 2 * 1.001 <= 2.5  # the polynomial kernel is the one used
        cell = np.clip(np.floor((X - ((lo + hi) / 2 - 2 ** L * side / 2)) / side), 0, 2 ** L - 1)
        # largest neighbour-pair u actually present
        from scipy.spatial import cKDTree
        pr = cKDTree(X).query_pairs(2 * np.sqrt(3) * side, output_type="ndarray")
        nb = np.all(np.abs(cell[pr[:, 0]] - cell[pr[:, 1]]) <= 1, axis=1)
        umax = (k * np.linalg.norm(X[pr[nb, 0]] - X[pr[nb, 1]], axis=1)).max() ** 2
        assert umax > 2.35
        s = synthetic.random_density(plan.n, seed=8)
        near, info = oracle.fmm(X, W, k, s, leaf_max=64, p_fixed=4, parts=1)
        assert info[0] == L
        assert rel(_apply(plan, s, parts=1), near) < 1e-5
    finally:
        plan.close()


def test_correction_against_oracle(c1):
    C = oracle.correction_csr(c1["V"], c1["F"], 1.0, c1["r"])
    assert C.nnz == c1["plan"].info()["corr_nnz"]
    assert rel(_apply(c1["plan"], c1["s"], parts=4), C @ c1["s"]) < 1e-5


def test_far_field_against_oracle_fmm(c1):
    X, W, _ = oracle.points(c1["V"], c1["F"])
    far, _ = oracle.fmm(X, W, 1.0, c1["s"], leaf_max=64, p_fixed=8, parts=2)
    got = _apply(c1["plan"], c1["s"], parts=2)
    # same octree and truncation: differences are rounding only
    assert np.linalg.norm(got - far) < 2e-6 * np.linalg.norm(c1["ref"])


def test_matvec_against_direct_sum_c1(c1):
    assert rel(_apply(c1["plan"], c1["s"]), c1["ref"]) < 1e-4


def test_matvec_host_buffers_match_device_matvec(c1):
    """hfmm_matvec_host (host buffers in and out, copies inside the call) against the
    device-pointer matvec and the oracle; one and three right-hand sides."""
    S = np.stack([synthetic.random_density(c1["plan"].n, seed=q) for q in range(3)])
    for R in (1, 3):
        h_in = torch.from_numpy(S[:R].reshape(-1).astype(np.complex64)).pin_memory()
        h_out = torch.full_like(h_in, complex(np.nan, np.nan)).pin_memory()
        c1["plan"].matvec_host(h_in, h_out, R)
        got = h_out.numpy().astype(np.complex128).reshape(R, -1)
        dev = _apply(c1["plan"], S[:R], nrhs=R)
        for q in range(R):
            assert rel(got[q], dev[q]) < 1e-6
    assert rel(got[0], c1["ref"]) < 1e-4


def test_direct_against_oracle(c1):
    d = _dev(c1["s"])
    o = torch.empty_like(d)
    c1["plan"].direct(d, o)
    assert rel(_host(o), c1["ref"]) < 1e-5


def test_multiple_right_hand_sides(c1):
    S = np.stack([synthetic.random_density(c1["plan"].n, seed=q) for q in range(3)])
    got = _apply(c1["plan"], S, nrhs=3)
    for q in range(3):
        assert rel(got[q], _apply(c1["plan"], S[q])) < 1e-6


def test_error_decreases_with_order(c1):
    errs = []
    for p in [4, 6, 8]:
        plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=p)
        try:
            errs.append(rel(_apply(plan, c1["s"]), c1["ref"]))
        finally:
            plan.close()
    assert errs[1] < errs[0] and errs[2] < errs[1]


@pytest.mark.parametrize("level,leaf", [(0, 4), (1, 16), (2, 20)])
def test_small_and_ragged_meshes(level, leaf):
    """Tiny meshes, leaves far below a warp, several octree levels."""
    V, F = synthetic.icosphere(level)
    k = 2.5
    plan = pkg.Plan(V, F, k, p_fixed=10, leaf_max=leaf)
    try:
        s = synthetic.random_density(plan.n, seed=level)
        ref = oracle.direct_matvec(V, F, k, oracle.near_radius(V, F, 1.0), s)
        assert rel(_apply(plan, s), ref) < 1e-4
    finally:
        plan.close()


def test_rhs_planewave(c1):
    d = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
    out = torch.empty(2 * c1["plan"].n, dtype=torch.complex64, device="cuda")
    c1["plan"].rhs_planewave(d, out)
    X, _, _ = oracle.points(c1["V"], c1["F"])
    got = _host(out).reshape(2, -1)
    for q in range(2):
        assert np.max(np.abs(got[q] - oracle.plane_wave(X, 1.0, d[q]))) < 1e-6


def test_solve_c1_against_dense_solution(c1):
    """GMRES(30) to 1e-4 on the small sphere.  The true residual, measured with
    the oracle's exact dense operator, is at most the tolerance plus the FMM's
    operator error; the solution error is bounded by cond(Z) times that."""
    plan = c1["plan"]
    b = _dev(np.zeros(plan.n))
    plan.rhs_planewave([0.0, 0.0, 1.0], b)
    x = torch.empty_like(b)
    st, its, rr = plan.solve(b, x)
    assert st == pkg.HFMM_OK and rr[0] <= 1e-4 and its[0] < 100
    assert plan.solver_info()["cycle_graph"] == 1  # each cycle one graph launch (while node)
    X, _, _ = oracle.points(c1["V"], c1["F"])
    Z = oracle.dense_Z(c1["V"], c1["F"], 1.0, c1["r"])
    bb = oracle.plane_wave(X, 1.0, (0, 0, 1))
    xg = _host(x)
    assert np.linalg.norm(Z @ xg - bb) / np.linalg.norm(bb) < 2e-4
    x_lu = np.linalg.solve(Z, bb)
    # cond(Z) ~ 60 here: 1e-4 residual plus ~1e-5 operator error -> ~1e-2 at worst
    assert rel(xg, x_lu) < 1e-2
    # Mie series (Sec. 6.4's analytic check): the dense solution sits at this mesh's
    # discretisation error (6.45e-3); a solve stopped at residual 1e-4 may sit up to
    # cond(Z) * 2e-4 ~ 1.2e-2 further (the C1 tolerance cannot resolve more).  The
    # equal-distance check is made on the tight solve below.
    qm = oracle.mie_surface_q(X, 1.0)
    e_lu, e_gpu = rel(x_lu, qm), rel(xg, qm)
    assert 5e-3 < e_lu < 7e-3
    assert e_gpu < e_lu + 60 * 2e-4


def test_solve_c1_matches_the_oracle_gmres(c1):
    """The converged GMRES solution against the oracle's: FP64 GMRES(30) to 1e-4 (the oracle's
    own implementation) on the oracle's operator, its FP64 FMM of the point part at the same
    order and tree plus its sparse correction.  The two operators differ by the GPU's FP32
    arithmetic (about 1e-6), so both solves take the same Krylov steps and stop at the same
    iteration; the solutions then agree to 1e-4."""
    plan = c1["plan"]
    V, F = c1["V"], c1["F"]
    b = _dev(np.zeros(plan.n))
    plan.rhs_planewave([0.0, 0.0, 1.0], b)
    x = torch.empty_like(b)
    st, its, rr = plan.solve(b, x)
    assert st == pkg.HFMM_OK
    X, W, _ = oracle.points(V, F)
    C = oracle.correction_csr(V, F, 1.0, c1["r"])

    def op(s):
        return oracle.fmm(X, W, 1.0, s, leaf_max=64, p_fixed=8, parts=3)[0] + C @ s

    bb = oracle.plane_wave(X, 1.0, (0, 0, 1))
    xo, it_o, rr_o, _ = oracle.gmres(op, bb, restart=30, tol=1e-4)
    assert abs(it_o - its[0]) <= 1
    assert rel(_host(x), xo) < 1e-4


def test_solve_tight_matches_dense_solution():
    """Higher order (operator error ~4e-7) and tolerance 5e-7 (an FP32 matvec
    cannot certify much less): solution within 1e-4 of the oracle's."""
    V, F = synthetic.sphere_mesh(2)
    plan = pkg.Plan(V, F, 1.0, p_fixed=12, tol=5e-7, leaf_max=32)
    try:
        b = _dev(np.zeros(plan.n))
        plan.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, its, rr = plan.solve(b, x)
        assert st == pkg.HFMM_OK
        X, _, _ = oracle.points(V, F)
        Z = oracle.dense_Z(V, F, 1.0, oracle.near_radius(V, F, 1.0))
        x_lu = np.linalg.solve(Z, oracle.plane_wave(X, 1.0, (0, 0, 1)))
        xg = _host(x)
        assert rel(xg, x_lu) < 1e-4
        # GPU and dense solutions equally far from the Mie series (discretisation error
        # 1.6e-2 on this mesh): their distances differ by less than 2e-4
        qm = oracle.mie_surface_q(X, 1.0)
        assert abs(rel(xg, qm) - rel(x_lu, qm)) < 2e-4
    finally:
        plan.close()


def test_solve_reports_non_convergence(c1):
    plan = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=6, max_iter=3)
    try:
        b = _dev(np.zeros(plan.n))
        plan.rhs_planewave([0.0, 0.0, 1.0], b)
        x = torch.empty_like(b)
        st, its, rr = plan.solve(b, x)
        assert st == pkg.HFMM_NOT_CONVERGED and its[0] == 3 and 1e-4 < rr[0] < 1.0
    finally:
        plan.close()


def test_zero_rhs_gives_zero_solution(c1):
    b = _dev(np.zeros(c1["plan"].n))
    x = _dev(np.ones(c1["plan"].n))
    st, its, rr = c1["plan"].solve(b, x)
    assert st == pkg.HFMM_OK and its[0] == 0 and np.all(_host(x) == 0)


@pytest.mark.parametrize("p", [3, 5, 7])
def test_tensor_core_m2l_against_simt_and_oracle(c1, p):
    """BF16x3 tcgen05 M2L ((p+1)^2 <= 64) against the FP32 SIMT form of the same
    plan and against the oracle's direct sum; p = 5 has (p+1)^2 = 36, not a
    multiple of 8 (element-wise operand staging)."""
    tc = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=p, m2l_tensor=1)
    simt = pkg.Plan(c1["V"], c1["F"], 1.0, p_fixed=p, m2l_tensor=0)
    try:
        far_tc = _apply(tc, c1["s"], parts=2)
        far_simt = _apply(simt, c1["s"], parts=2)
        assert tc.device_status() == pkg.HFMM_OK
        # BF16 split in three products: ~1e-5 relative to the far field
        assert np.linalg.norm(far_tc - far_simt) < 3e-5 * np.linalg.norm(far_simt)
        e_tc = rel(_apply(tc, c1["s"]), c1["ref"])
        e_simt = rel(_apply(simt, c1["s"]), c1["ref"])
        assert e_tc < e_simt + 2e-6
        if p == 7:
            assert e_tc < 1e-4
    finally:
        tc.close()
        simt.close()
