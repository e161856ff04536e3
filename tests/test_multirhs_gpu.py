"""Several right-hand sides on one mesh: clones share the mesh data and are
solved together in one batched graph launch.  Small 3-D case against the
oracle; the full 16^3 p = 7 workload with 32 right-hand sides checked on
sampled right-hand sides through the oracle's own FP64 operator (the true
residual), which holds at any size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solve as osolve  # noqa: E402
from oracle.discretize import Level, lift  # noqa: E402
from oracle.multigrid import Hierarchy  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
def test_multirhs_3d_matches_oracle(prec):
    wl = inputs.random3d((3, 3, 2), 5, amp=0.15, seed=31, nrhs=4)
    prob, coords = glls.problem_for(wl)
    F = wl.sample_rhs(coords).reshape(wl.nrhs, -1)
    g = wl.sample_dirichlet(coords).ravel()
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=prec)
    U, stats, clones = glls.solve_multi(prob, F, g, o)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    ref = osolve.solve(wl, gamma=1, alpha=0.5, tol=1e-10, hierarchy=Hierarchy(fine, restriction="transpose"))
    for j in range(wl.nrhs):
        r = ref.u[j].ravel()
        assert np.abs(U[j] - r).max() <= (1e-9 if prec == glls.PREC_FP64 else 1e-8) * np.abs(r).max()
        assert stats[j].rel_residual <= 1e-10
    # the clones keep the shared mesh data alive after the original is gone
    prob.close()
    U2, _, _ = glls.solve_multi(clones[0], F[1:], g, o, clones=clones[1:])
    np.testing.assert_allclose(U2, U[1:], rtol=0, atol=1e-10 * np.abs(U).max())
    for c in clones:
        c.close()


def test_terrain3d_full_size_32_rhs_true_residual():
    """16^3 elements, p = 7 (1,442,897 nodes), 32 right-hand sides solved
    together, mixed precision; true FP64 residual of sampled right-hand
    sides computed by the oracle's operator."""
    wl = inputs.terrain3d()
    prob, coords = glls.problem_for(wl)
    info = prob.info
    assert prob.N == 113 ** 3 and [info.order[l] for l in range(info.levels)] == [1, 3, 7]
    F = wl.sample_rhs(coords).reshape(wl.nrhs, -1)
    g = np.zeros(prob.N)
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=glls.PREC_MIXED)
    U, stats, clones = glls.solve_multi(prob, F, g, o)
    assert all(st.status == glls.OK and st.rel_residual <= 1e-10 for st in stats)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    for j in (0, 17, 31):
        f0, v = lift(fine, F[j].reshape(fine.shape), g.reshape(fine.shape))
        w = U[j].reshape(fine.shape) - v
        res = np.linalg.norm((f0 - fine.apply(w))[fine.interior]) / np.linalg.norm(f0[fine.interior])
        assert res <= 2e-10, (j, res)
    for c in clones:
        c.close()
    prob.close()
