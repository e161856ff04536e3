"""Coloured direct stiffness summation (GLLS_SUM_COLORED, the sum over elements
of Sec. 2 taken colour by colour in a fixed order): the apply equals the
oracle's and the atomic summation's to rounding, and a solve gives the same
bits on every run, alone, in a graph-branch batch and in the serving loop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.discretize import Level  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402

TOL64 = 1e-12
TOL32 = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# odd and even element counts per axis (colours of different sizes, empty
# colours along an axis of one element), a single element (one colour), the
# generic order range (p = 17) and 3-D edges and vertices shared by 4 and 8
# elements
APPLY_CASES = [
    ("2d_5x4_p6", lambda: inputs.random2d((5, 4), 6, amp=0.1, seed=81)),
    ("2d_7x1_p8", lambda: inputs.random2d((7, 1), 8, amp=0.1, seed=82)),
    ("2d_3x3_p17", lambda: inputs.random2d((3, 3), 17, amp=0.05, seed=83)),
    ("2d_single_p8", lambda: inputs.table1_problem3(8)),
    ("3d_3x2x3_p5", lambda: inputs.random3d((3, 2, 3), 5, amp=0.1, seed=84)),
    ("3d_3x3x3_p7", lambda: inputs.random3d((3, 3, 3), 7, amp=0.1, seed=85)),
    ("3d_2x1x3_p3", lambda: inputs.random3d((2, 1, 3), 3, amp=0.15, seed=86)),
]


@pytest.mark.parametrize("name,mk", APPLY_CASES, ids=[c[0] for c in APPLY_CASES])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_colored_apply_matches_oracle_and_atomic(name, mk, dtype):
    wl = mk()
    col, coords = glls.problem_for(wl, summation=glls.SUM_COLORED)
    ato, _ = glls.problem_for(wl)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    rng = np.random.default_rng(7)
    x = np.where(fine.interior, rng.standard_normal(fine.shape), 0.0)
    L = col.levels - 1
    xd = torch.tensor(x.ravel(), dtype=dtype, device="cuda")
    ys = []
    for prob in (col, col, ato):
        y = torch.zeros(fine.N, dtype=dtype, device="cuda")
        prob.apply(L, xd, y)
        torch.cuda.synchronize()
        ys.append(y.double().cpu().numpy())
    ref = fine.apply(x).ravel()
    tol = TOL64 if dtype == torch.float64 else TOL32
    if wl.order > 16:
        tol *= 9      # contraction rounding grows with the GLL derivative entries (~p^2)
    assert _rel(ys[0], ref) < tol
    assert np.array_equal(ys[0], ys[1])          # same bits on a second run
    assert _rel(ys[0], ys[2]) < tol              # atomic summation: same values to rounding
    col.close()
    ato.close()


SOLVE_MIX = [inputs.random2d((9, 7), 6, amp=0.1, seed=91), inputs.random2d((12, 10), 8, amp=0.1, seed=92),
             inputs.random3d((3, 3, 2), 4, amp=0.1, seed=93), inputs.random2d((5, 6), 5, amp=0.1, seed=94)]


def _colored(wl):
    prob, coords = glls.problem_for(wl, summation=glls.SUM_COLORED)
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    prob.set_rhs(f)
    prob.set_dirichlet(g)
    return prob, coords, f, g


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
def test_colored_solves_same_bits_alone_repeated_and_batched(prec):
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec, max_iter=300)
    probs = [_colored(wl)[0] for wl in SOLVE_MIX]
    alone, its = [], []
    for p in probs:
        u = np.zeros(p.N)
        st = p.solve(u, o)
        assert st.status == glls.OK and st.rel_residual <= 1e-10
        u2 = np.zeros(p.N)
        st2 = p.solve(u2, o)
        assert np.array_equal(u, u2) and st2.iterations == st.iterations
        alone.append(u)
        its.append(st.iterations)
    for _ in range(2):
        outs = [np.zeros(p.N) for p in probs]
        stats = glls.solve_batch(probs, outs, o)
        for u, ub, st, k in zip(alone, outs, stats, its):
            assert np.array_equal(ub, u)
            assert st.iterations == k and st.status == glls.OK
    # the work-list kernels sum with atomics: such a batch is refused
    with pytest.raises(glls.GllsError) as ei:
        glls.solve_batch(probs, [np.zeros(p.N) for p in probs], o, worklist=True)
    assert ei.value.status == glls.ERR_INVALID
    for p in probs:
        p.close()


def test_colored_solve_matches_atomic_solve():
    """Same iterate to the solver tolerance whichever summation: the order of
    the seam additions changes only the rounding."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_FP64)
    wl = SOLVE_MIX[1]
    col, coords, f, g = _colored(wl)
    ato, _ = glls.problem_for(wl)
    ato.set_rhs(f)
    ato.set_dirichlet(g)
    uc, ua = np.zeros(col.N), np.zeros(ato.N)
    sc, sa = col.solve(uc, o), ato.solve(ua, o)
    assert abs(sc.iterations - sa.iterations) <= 1
    assert _rel(uc, ua) < 1e-9
    col.close()
    ato.close()


def test_server_colored_results_same_bits_alone_and_in_the_mix():
    """Concurrent requests on registered coloured meshes (clones, several
    slots, grouping into multi-right-hand-side solves switched on) return
    exactly the bits of the solve alone."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    reqs = [_colored(wl) for wl in SOLVE_MIX[:3]]
    alone = []
    for prob, coords, f, g in reqs:
        u = np.zeros(prob.N)
        assert prob.solve(u, o).status == glls.OK
        alone.append(u)
        prob.close()
    srv = glls.Server(budget_bytes=8 << 30, slots=4)
    srv.set_max_group(4)
    ids = [srv.register(wl.dim, wl.nelem, wl.order, c, summation=glls.SUM_COLORED)
           for wl, (_, c, _, _) in zip(SOLVE_MIX, reqs)]
    outs, tickets = [], []
    for _ in range(4):
        for k, (_, _, f, g) in enumerate(reqs):
            out = np.full(f.size, np.nan)
            outs.append((k, out))
            tickets.append(srv.submit_mesh(ids[k], f, g, o, out))
    for t in tickets:
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK
    srv.close()
    for k, out in outs:
        assert np.array_equal(out, alone[k])


def test_bad_summation_is_refused():
    wl = inputs.random2d((3, 3), 4, amp=0.1, seed=95)
    with pytest.raises(glls.GllsError) as ei:
        glls.problem_for(wl, summation=2)
    assert ei.value.status == glls.ERR_INVALID


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("mk", [lambda: inputs.random2d((7, 5), 6, amp=0.1, seed=96, nrhs=3),
                                lambda: inputs.random3d((3, 2, 2), 5, amp=0.1, seed=97, nrhs=4)],
                         ids=["2d_7x5_p6_x3", "3d_3x2x2_p5_x4"])
def test_colored_nrhs_solve_same_bits_as_single_solves(mk, prec):
    """With coloured summation every kernel of a multi-right-hand-side solve
    does, for each right-hand side, the arithmetic of a single solve in the
    same order (right-hand sides only add CTAs): each result is the bits of
    its single solve."""
    wl = mk()
    prob, coords = glls.problem_for(wl, nrhs=wl.nrhs, summation=glls.SUM_COLORED)
    F = np.ascontiguousarray(wl.sample_rhs(coords).reshape(wl.nrhs, -1))
    g = wl.sample_dirichlet(coords).ravel()
    prob.set_rhs(F)
    prob.set_dirichlet(g)
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec)
    U = np.zeros((wl.nrhs, prob.N))
    stats = prob.solve(U, o)
    single = glls.problem_for(wl, summation=glls.SUM_COLORED)[0]
    single.set_dirichlet(g)
    for j in range(wl.nrhs):
        single.set_rhs(F[j])
        u1 = np.zeros(prob.N)
        s1 = single.solve(u1, o)
        assert stats[j].iterations == s1.iterations
        assert np.array_equal(U[j], u1), (j, np.abs(U[j] - u1).max())
    single.close()
    prob.close()


def test_server_groups_colored_requests_with_single_solve_bits():
    """One slot and grouping on: queued requests of a coloured mesh are solved
    together as multi-right-hand-side solves, and each result is the bits of
    its right-hand side solved alone."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    wl = SOLVE_MIX[1]
    prob, coords, f, g = _colored(wl)
    fs = [f * (1.0 + 0.3 * j) - 0.1 * j for j in range(6)]
    alone = []
    for fk in fs:
        prob.set_rhs(fk)
        u = np.zeros(prob.N)
        assert prob.solve(u, o).status == glls.OK
        alone.append(u)
    prob.close()
    srv = glls.Server(budget_bytes=8 << 30, slots=1)
    srv.set_max_group(4)
    mid = srv.register(wl.dim, wl.nelem, wl.order, coords, summation=glls.SUM_COLORED)
    outs = [np.full(f.size, np.nan) for _ in fs]
    tickets = [srv.submit_mesh(mid, fk, g, o, out) for fk, out in zip(fs, outs)]
    groups = []
    for t in tickets:
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK
        groups.append(stats.group)
    srv.close()
    assert max(groups) > 1, groups
    for out, u in zip(outs, alone):
        assert np.array_equal(out, u)
