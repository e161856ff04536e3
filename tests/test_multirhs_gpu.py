"""Several right-hand sides on one mesh, two ways: one problem created with
nrhs right-hand sides, whose kernels process all of them per launch; and
clones that share the mesh data, solved together in one batched graph
launch.  Small cases against the oracle and against single solves; the full
16^3 p = 7 workload with 32 right-hand sides checked on sampled right-hand
sides through the oracle's own FP64 operator (the true residual), which
holds at any size."""
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


MULTI = [("2d_7x5_p6", lambda: inputs.random2d((7, 5), 6, amp=0.1, seed=33, nrhs=3)),
         ("3d_3x3x2_p5", lambda: inputs.random3d((3, 3, 2), 5, amp=0.15, seed=31, nrhs=4)),
         ("2d_4x3_p1", lambda: inputs.random2d((4, 3), 1, amp=0.05, seed=34, nrhs=3)),
         ("3d_2x3x2_p3", lambda: inputs.random3d((2, 3, 2), 3, amp=0.1, seed=35, nrhs=5))]


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,mk", MULTI, ids=[m[0] for m in MULTI])
def test_nrhs_problem_equals_single_solves(name, mk, prec):
    """A problem with nrhs right-hand sides gives, for each, the solution and
    iteration count of a one-right-hand-side solve of it, and the oracle's."""
    wl = mk()
    prob, coords = glls.problem_for(wl, nrhs=wl.nrhs)
    F = wl.sample_rhs(coords).reshape(wl.nrhs, -1)
    g = wl.sample_dirichlet(coords).ravel()
    prob.set_rhs(np.ascontiguousarray(F))
    prob.set_dirichlet(g)
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec)
    U = np.zeros((wl.nrhs, prob.N))
    stats = prob.solve(U, o)
    single = glls.problem_for(wl)[0]
    single.set_dirichlet(g)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    ref = osolve.solve(wl, gamma=1, alpha=2.0 / 3.0, tol=1e-10, hierarchy=Hierarchy(fine, restriction="transpose"))
    for j in range(wl.nrhs):
        single.set_rhs(F[j])
        u1 = np.zeros(prob.N)
        s1 = single.solve(u1, o)
        assert stats[j].status == glls.OK and stats[j].rel_residual <= 1e-10
        assert stats[j].iterations == s1.iterations, (j, stats[j].iterations, s1.iterations)
        assert np.abs(U[j] - u1).max() <= 1e-11 * np.abs(u1).max(), j
        r = ref.u[j].ravel()
        assert np.abs(U[j] - r).max() <= (1e-9 if prec == glls.PREC_FP64 else 1e-8) * np.abs(r).max()
    single.close()
    prob.close()


def test_nrhs_each_right_hand_side_stops_on_its_own():
    """Zero data stops at once with u = 0, a NaN right-hand side breaks down,
    a scaled copy takes the same iterations; the others are unaffected and
    the call reports the worst status."""
    wl = inputs.random2d((6, 5), 5, amp=0.1, seed=36, nrhs=1)
    prob, coords = glls.problem_for(wl, nrhs=4)
    f = wl.sample_rhs(coords).reshape(-1)
    F = np.stack([f, np.zeros_like(f), 1e6 * f, f.copy()])
    nx = prob.level_shape(prob.levels - 1)[-1]
    F[3, 10 * nx + 10] = np.nan          # an interior node (boundary values of f are not used)
    prob.set_rhs(np.ascontiguousarray(F))
    prob.set_dirichlet(np.zeros(prob.N))
    U = np.zeros((4, prob.N))
    stats = prob.solve(U, glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED),
                       raise_on_error=False)
    assert stats[0].status == glls.OK and stats[0].iterations > 3
    assert stats[1].status == glls.OK and stats[1].iterations == 0 and not U[1].any()
    assert stats[2].status == glls.OK and abs(stats[2].iterations - stats[0].iterations) <= 1
    assert np.abs(U[2] - 1e6 * U[0]).max() <= 1e-8 * np.abs(U[2]).max()
    assert stats[3].status == glls.ERR_BREAKDOWN
    with pytest.raises(glls.GllsError) as ei:
        prob.solve(U, glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED))
    assert ei.value.status == glls.ERR_BREAKDOWN
    # several right-hand sides need the device-loop graph and FCG / PCG
    with pytest.raises(glls.GllsError):
        prob.solve(U, glls.opts(use_graph=1))
    prob.close()


def test_terrain3d_full_size_32_rhs_in_one_problem():
    """The 3-D workload's 32 right-hand sides as one problem with nrhs = 32
    (every kernel launch covers all of them): each converges to 1e-10 and
    its true FP64 residual, by the oracle's operator, agrees."""
    wl = inputs.terrain3d()
    prob, coords = glls.problem_for(wl, nrhs=wl.nrhs)
    F = np.ascontiguousarray(wl.sample_rhs(coords).reshape(wl.nrhs, -1))
    g = np.zeros(prob.N)
    prob.set_rhs(F)
    prob.set_dirichlet(g)
    U = np.zeros((wl.nrhs, prob.N))
    stats = prob.solve(U, glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED))
    assert all(st.status == glls.OK and st.rel_residual <= 1e-10 for st in stats)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    for j in (0, 17, 31):
        f0, v = lift(fine, F[j].reshape(fine.shape), g.reshape(fine.shape))
        w = U[j].reshape(fine.shape) - v
        res = np.linalg.norm((f0 - fine.apply(w))[fine.interior]) / np.linalg.norm(f0[fine.interior])
        assert res <= 2e-10, (j, res)
    prob.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("dims", [((5, 4), 8), ((3, 3, 2), 7), ((4, 3, 2), 3)], ids=["2d_p8", "3d_p7", "3d_p3"])
def test_apply_multi_equals_single_applies(dtype, dims):
    """glls_apply_multi on k stacked vectors (one launch, the operator read
    once) equals k single applies, every level."""
    nelem, p = dims
    wl = inputs.random2d(nelem, p, amp=0.1, seed=41) if len(nelem) == 2 else inputs.random3d(nelem, p, seed=41)
    prob, _ = glls.problem_for(wl)
    k = 5
    gen = torch.Generator(device="cuda").manual_seed(7)
    for level in range(prob.levels):
        n = int(np.prod(prob.level_shape(level)))
        X = torch.randn(k * n, dtype=dtype, device="cuda", generator=gen)
        Y = torch.zeros_like(X)
        prob.apply_multi(level, X, Y, k)
        for j in range(k):
            y1 = torch.zeros(n, dtype=dtype, device="cuda")
            prob.apply(level, X[j * n:(j + 1) * n].contiguous(), y1)
            scale = float(y1.abs().max())
            tol = 1e-13 if dtype == torch.float64 else 2e-6
            assert float((Y[j * n:(j + 1) * n] - y1).abs().max()) <= tol * scale
    prob.close()
