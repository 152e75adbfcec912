"""Off-surface evaluation: the single-layer potential of a density at observation
points away from the surface, against the oracle's FP64 definition (1e-5 relative),
and end to end for the sound-soft sphere: solve for the surface density, evaluate
-field at 4 m (the paper's observation distance) and compare with the exact Mie
scattered field; the error is the discretisation's and falls under mesh refinement."""
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


def _field(plan, dens, T):
    d = torch.from_numpy(np.ascontiguousarray(dens).astype(np.complex64)).cuda()
    o = torch.empty(T.shape[0], dtype=torch.complex64, device="cuda")
    plan.field(d, T, o)
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.complex128)


def test_field_against_oracle_definition():
    V, F = synthetic.sphere_mesh(3)
    k = 3.0
    plan = pkg.Plan(V, F, k, p_fixed=6)
    try:
        X, W, _ = oracle.points(V, F)
        s = synthetic.random_density(plan.n, seed=8)
        rng = np.random.default_rng(2)
        U = rng.standard_normal((333, 3))  # 333: a ragged last block of targets
        U /= np.linalg.norm(U, axis=1, keepdims=True)
        T = U * rng.uniform(1.5, 4.0, size=(333, 1))
        assert _rel(_field(plan, s, T), oracle.field_direct(X, W, k, s, T)) < 1e-5
    finally:
        plan.close()


def test_scattered_field_at_4m_against_mie():
    k = 2.0
    d = np.asarray(synthetic.fibonacci_directions(64, seed=1)).reshape(64, 3)
    T = 4.0 * d
    exact = oracle.mie_scattered(T, k)
    errs = []
    for level in (3, 4):
        V, F = synthetic.sphere_mesh(level)
        plan = pkg.Plan(V, F, k, p_fixed=8, tol=1e-6)
        try:
            b = torch.empty(plan.n, dtype=torch.complex64, device="cuda")
            plan.rhs_planewave([0.0, 0.0, 1.0], b)
            x = torch.empty_like(b)
            st, _, _ = plan.solve(b, x)
            assert st == pkg.HFMM_OK
            o = torch.empty(64, dtype=torch.complex64, device="cuda")
            plan.field(x, T, o)
            torch.cuda.synchronize()
            errs.append(_rel(-o.cpu().numpy().astype(np.complex128), exact))
        finally:
            plan.close()
    assert errs[0] < 2e-2 and errs[1] < 0.6 * errs[0]
