"""Batched right-hand sides: hfmm_matvec with nrhs = 2..64 runs one batched matvec
(expansions [box][rhs][P], the near-field Green's function evaluated once for all
right-hand sides, translations with one work item per box pair and nrhs columns),
replayed from a captured CUDA graph.

Tolerances (relative 2-norm per right-hand side):
  batched vs the single right-hand-side path of the same plan   5e-6  (FP32; the near field sums ~400
                                                                 terms per point in another order)
  batched vs the oracle's direct summation                      1e-4  (the matvec bar)
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dens(n, nrhs, seed):
    return np.stack([synthetic.random_density(n, seed=seed + r) for r in range(nrhs)])  # [nrhs][n]


def _batched(plan, S):
    d = torch.from_numpy(np.ascontiguousarray(S).astype(np.complex64).reshape(-1)).cuda()
    o = torch.full_like(d, complex(np.nan, np.nan))
    plan.matvec(d, o, S.shape[0])
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128).reshape(S.shape)


def _single(plan, S):
    out = []
    for s in S:
        d = torch.from_numpy(s.astype(np.complex64)).cuda()
        o = torch.empty_like(d)
        plan.matvec(d, o, 1)
        torch.cuda.synchronize()
        out.append(o.cpu().numpy().astype(np.complex128))
    return np.stack(out)


@pytest.fixture(scope="module")
def small():
    V, F = synthetic.sphere_mesh(3)
    yield V, F


@pytest.mark.parametrize("p,nrhs", [(7, 5), (7, 64), (8, 3), (5, 37)])
def test_batched_matches_single_and_oracle(small, p, nrhs):
    """p = 7: P = 64 on the tensor cores; p = 8: P = 81 (SIMT translations, two
    coefficient tiles in the batched P2M); p = 5: P = 36 (element-wise operand staging)."""
    V, F = small
    plan = pkg.Plan(V, F, 1.0, p_fixed=p, leaf_max=64)
    try:
        S = _dens(plan.n, nrhs, seed=10)
        got = _batched(plan, S)
        assert plan.device_status() == pkg.HFMM_OK
        assert np.all(np.isfinite(got))
        ref1 = _single(plan, S)
        for r in range(nrhs):
            assert _rel(got[r], ref1[r]) < 5e-6, r
        rr = oracle.near_radius(V, F, plan.cfg.near_factor)
        for r in (0, nrhs - 1):
            assert _rel(got[r], oracle.direct_matvec(V, F, 1.0, rr, S[r])) < (1e-4 if p >= 7 else 1e-2)
    finally:
        plan.close()


def test_more_than_64_rhs_and_graph_replay(small):
    """70 right-hand sides run as 64 + 6; repeated calls replay the captured graph,
    and new buffers re-capture it."""
    V, F = small
    plan = pkg.Plan(V, F, 1.0, p_fixed=7)
    try:
        S = _dens(plan.n, 70, seed=40)
        a = _batched(plan, S)
        b = _batched(plan, S)  # new tensors: new graph
        ref1 = _single(plan, S[[0, 63, 64, 69]])
        for q, r in enumerate((0, 63, 64, 69)):
            assert _rel(a[r], ref1[q]) < 5e-6
        # reductions into the expansions run in any order: equal up to FP32 rounding
        for r in range(70):
            assert _rel(b[r], a[r]) < 5e-6
        d = torch.from_numpy(np.ascontiguousarray(S[:8]).astype(np.complex64).reshape(-1)).cuda()
        o = torch.empty_like(d)
        outs = []
        for _ in range(3):  # same buffers: replays
            plan.matvec(d, o, 8)
            torch.cuda.synchronize()
            outs.append(o.cpu().numpy())
        assert _rel(outs[2].astype(np.complex128), outs[1].astype(np.complex128)) < 5e-6
        assert _rel(outs[0].astype(np.complex128).reshape(8, -1)[5], _single(plan, S[5:6])[0]) < 5e-6
    finally:
        plan.close()


def test_batched_planewaves_491k_sampled_rows():
    """The batched configuration: N = 491,520, k = 10, 64 plane waves from a seeded
    Fibonacci sphere; every right-hand side against the single path on all points,
    four against the oracle on sampled rows."""
    V, F = synthetic.workload_mesh("sphere_163840")
    k = 10.0
    plan = pkg.Plan(V, F, k)
    try:
        dirs = synthetic.fibonacci_directions(64, seed=0)
        b = torch.empty(64 * plan.n, dtype=torch.complex64, device="cuda")
        plan.rhs_planewave(np.asarray(dirs).reshape(64, 3), b)
        torch.cuda.synchronize()
        S = b.cpu().numpy().astype(np.complex128).reshape(64, plan.n)
        got = _batched(plan, S)
        assert plan.device_status() == pkg.HFMM_OK
        ref1 = _single(plan, S[[0, 21, 42, 63]])
        for q, r in enumerate((0, 21, 42, 63)):
            assert _rel(got[r], ref1[q]) < 5e-6
        rr = oracle.near_radius(V, F, plan.cfg.near_factor)
        rng = np.random.default_rng(9)
        rows = np.unique(np.concatenate([rng.choice(plan.n, 48, replace=False), [0, plan.n - 1]]))
        for r in (0, 31, 63):
            ref = oracle.direct_rows(V, F, k, rr, rows, S[r])
            assert _rel(got[r][rows], ref) < 1e-4
    finally:
        plan.close()


def _dense_setup(V, F, k):
    X, _, _ = oracle.points(V, F)
    Z = oracle.dense_Z(V, F, k, oracle.near_radius(V, F, 1.0))
    return X, Z


def test_batched_solve_against_dense_solutions(small):
    """hfmm_solve with 5 right-hand sides runs 5 GMRES(30) processes in lockstep on
    batched matvecs. Each solution meets the single-RHS solve's criteria: true residual
    under the oracle's dense operator <= 2e-4, distance to the dense-LU solution <= 1e-2
    (cond(Z) ~ 60); the second right-hand side is zero (zero solution, 0 iterations)."""
    V, F = small
    plan = pkg.Plan(V, F, 1.0, p_fixed=8, leaf_max=64, restart=30)
    try:
        dirs = np.asarray(synthetic.fibonacci_directions(5, seed=2)).reshape(5, 3)
        b = torch.empty(5 * plan.n, dtype=torch.complex64, device="cuda")
        plan.rhs_planewave(dirs, b)
        b.view(5, plan.n)[1].zero_()
        x = torch.full_like(b, complex(np.nan, np.nan))
        st, its, rr = plan.solve(b, x, 5)
        assert st == pkg.HFMM_OK
        torch.cuda.synchronize()
        xs = x.cpu().numpy().astype(np.complex128).reshape(5, plan.n)
        bs = b.cpu().numpy().astype(np.complex128).reshape(5, plan.n)
        assert its[1] == 0 and np.all(xs[1] == 0)
        X, Z = _dense_setup(V, F, 1.0)
        for r in (0, 2, 3, 4):
            assert rr[r] <= 1e-4 and 0 < its[r] < 100
            assert _rel(Z @ xs[r], bs[r]) < 2e-4
            assert _rel(xs[r], np.linalg.solve(Z, bs[r])) < 1e-2
    finally:
        plan.close()


def test_batched_solve_matches_single_solves_tight():
    """At p = 12 and tolerance 5e-7 the lockstep solves and one-at-a-time solves of the
    same right-hand sides agree to 1e-4, and each is within 1e-4 of the dense-LU solution."""
    V, F = synthetic.sphere_mesh(2)
    plan = pkg.Plan(V, F, 1.0, p_fixed=12, tol=5e-7, leaf_max=32)
    try:
        dirs = np.asarray(synthetic.fibonacci_directions(3, seed=4)).reshape(3, 3)
        b = torch.empty(3 * plan.n, dtype=torch.complex64, device="cuda")
        plan.rhs_planewave(dirs, b)
        xb = torch.empty_like(b)
        st, its, rr = plan.solve(b, xb, 3)
        assert st == pkg.HFMM_OK
        X, Z = _dense_setup(V, F, 1.0)
        bs = b.cpu().numpy().astype(np.complex128).reshape(3, plan.n)
        xbs = xb.cpu().numpy().astype(np.complex128).reshape(3, plan.n)
        for r in range(3):
            b1 = b.view(3, plan.n)[r].clone()
            x1 = torch.empty_like(b1)
            s1, _, _ = plan.solve(b1, x1)
            assert s1 == pkg.HFMM_OK
            x1h = x1.cpu().numpy().astype(np.complex128)
            assert _rel(xbs[r], x1h) < 1e-4
            assert _rel(xbs[r], np.linalg.solve(Z, bs[r])) < 1e-4
    finally:
        plan.close()
