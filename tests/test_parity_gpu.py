"""Parity of every hot-path step of the CUDA library (through the C ABI)
against the FP64 CPU oracle, element by element on the same seeded inputs.

Tolerances: FP64 kernels 1e-12 relative to the largest output entry (only the
summation order differs); FP32 kernels 5e-5 (single-precision rounding of
O(p) term contractions); whole FP64 solves 1e-9 relative with iteration
counts within one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solve as osolve  # noqa: E402
from oracle.discretize import Level, lift  # noqa: E402
from oracle.multigrid import Hierarchy  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402

TOL64 = 1e-12
TOL32 = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


SMOOTHERS = {"gll": glls.SMOOTHER_GLL, "fem": glls.SMOOTHER_FEM, "gll_band1": glls.SMOOTHER_GLL_BAND1}
RESTRICTIONS = {"transpose": glls.RESTRICT_TRANSPOSE, "interp": glls.RESTRICT_INTERP}


def make(wl, smoother="gll", restriction="transpose"):
    prob, coords = glls.problem_for(wl, SMOOTHERS[smoother], RESTRICTIONS[restriction])
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    return prob, Hierarchy(fine, smoother=smoother, restriction=restriction), coords


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def interior_field(lv, seed):
    return np.where(lv.interior, inputs.random_field(lv.shape, seed), 0.0)


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    ("2d_3x2_p4", lambda: inputs.random2d((3, 2), 4, amp=0.1, seed=1), "gll", "transpose"),
    ("2d_5x3_p8_fem", lambda: inputs.random2d((5, 3), 8, amp=0.15, seed=2), "fem", "transpose"),
    ("2d_7x5_p6", lambda: inputs.random2d((7, 5), 6, amp=0.1, seed=3), "gll", "transpose"),
    ("2d_4x4_p3_interp", lambda: inputs.random2d((4, 4), 3, amp=0.05, seed=4), "gll", "interp"),
    ("2d_single_p8", lambda: inputs.table1_problem3(8), "gll", "interp"),
    ("2d_single_p11_fem", lambda: inputs.table1_problem3(11), "fem", "interp"),
    ("3d_2x3x2_p3", lambda: inputs.random3d((2, 3, 2), 3, amp=0.15, seed=5), "gll", "transpose"),
    ("3d_3x2x2_p5_fem", lambda: inputs.random3d((3, 2, 2), 5, amp=0.1, seed=6), "fem", "transpose"),
    # limits: the highest order (generic apply above p = 16), lines longer than
    # the FP64 warp kernel takes (527 unknowns: shared-memory line kernel in
    # FP64, 32 unknowns per lane in FP32), the largest specialised orders.
    # The fifth entry scales the FP64 tolerance: the rounding of the
    # contractions relative to the largest output grows with the GLL
    # derivative entries (~p^2: (24/8)^2 = 9 at p = 24).  The long-line grid
    # has square elements: on stretched deformed elements single line systems
    # reach condition numbers of 1e4-1e5 and the two CR implementations then
    # differ by about that times the unit roundoff.
    ("2d_single_p24_generic", lambda: inputs.table1_problem3(24), "gll", "interp", 9),
    # (FP64 apply / lifting on this 280k-node grid: 2.1e-12 / 2.4e-12 relative to the largest output,
    # summation-order rounding of sums whose term magnitudes exceed that output by ~1e3)
    ("2d_66x66_p8_long_lines", lambda: inputs.random2d((66, 66), 8, amp=0.1, seed=13), "gll", "transpose", 4),
    ("3d_2x2x2_p8", lambda: inputs.random3d((2, 2, 2), 8, amp=0.1, seed=14), "gll", "transpose"),
    ("2d_3x2_p16", lambda: inputs.random2d((3, 2), 16, amp=0.1, seed=15), "gll", "transpose", 4),
    # the band-1 reading of the GLL line systems (band-1 warp kernel), 2-D and 3-D
    ("2d_7x5_p6_band1", lambda: inputs.random2d((7, 5), 6, amp=0.1, seed=3), "gll_band1", "transpose"),
    ("3d_2x3x2_p3_band1", lambda: inputs.random3d((2, 3, 2), 3, amp=0.15, seed=5), "gll_band1", "transpose"),
    # line blocks: more than 64 elements along x (vertex systems of 65..128
    # unknowns), odd orders 3..7 with 3-D faces and edges shared by 2-4 elements
    ("2d_70x3_p4_blocks", lambda: inputs.random2d((70, 3), 4, amp=0.1, seed=17), "gll", "transpose"),
    ("3d_3x2x4_p7_blocks", lambda: inputs.random3d((3, 2, 4), 7, amp=0.1, seed=18), "gll", "transpose"),
    ("3d_2x2x2_p5_blocks", lambda: inputs.random3d((2, 2, 2), 5, amp=0.15, seed=19), "gll", "transpose"),
    # orders 9..12: compile-time line-block instances with the operators in shared memory
    ("2d_4x3_p10_blocks", lambda: inputs.random2d((4, 3), 10, amp=0.1, seed=21), "gll", "transpose"),
    ("2d_3x2_p12_blocks", lambda: inputs.random2d((3, 2), 12, amp=0.15, seed=22), "gll", "transpose"),
    ("2d_single_p9_blocks", lambda: inputs.table1_problem3(9), "gll", "interp"),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _, mk, sm, rs = request.param[:4]
    scale = request.param[4] if len(request.param) > 4 else 1
    wl = mk()
    prob, h, coords = make(wl, sm, rs)
    yield wl, prob, h, coords, scale
    prob.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_apply(case, dtype):
    wl, prob, h, _, scale = case
    tol = TOL64 * scale if dtype == torch.float64 else TOL32
    for l, lv in enumerate(h.levels):
        x = interior_field(lv, 10 + l)
        y = torch.zeros(lv.N, dtype=dtype, device="cuda")
        prob.apply(l, dev(x, dtype), y)
        ref = lv.apply(x)
        assert relerr(host(y).reshape(lv.shape), ref) < tol, (l, relerr(host(y).reshape(lv.shape), ref))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_line_solve(case, dtype):
    wl, prob, h, _, scale = case
    tol = TOL64 * scale if dtype == torch.float64 else TOL32
    for l in range(1, len(h.levels)):
        lv = h.levels[l]
        for s in range(lv.dim):
            g = interior_field(lv, 20 + 3 * l + s)
            x = torch.zeros(lv.N, dtype=dtype, device="cuda")
            prob.line_solve(l, s, dev(g, dtype), x)
            ref = h.smoothers[l][s].apply_inverse(g)
            assert relerr(host(x).reshape(lv.shape), ref) < tol * 10, (l, s)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_smooth(case, dtype):
    wl, prob, h, _, scale = case
    tol = TOL64 * scale if dtype == torch.float64 else TOL32
    alpha = 0.5
    for l in range(1, len(h.levels)):
        lv = h.levels[l]
        for s in range(lv.dim):
            x0 = interior_field(lv, 40 + l)
            r = interior_field(lv, 50 + l)
            x = dev(x0, dtype)
            prob.smooth(l, s, alpha, dev(r, dtype), x)
            ref = h.smoothers[l][s].smooth(x0, r, alpha)
            assert relerr(host(x).reshape(lv.shape), ref) < tol * 10, (l, s)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_line_update_after_apply(case, dtype):
    """The smoothing step as two entry points: y = A x, then the line update
    x += alpha B_s^-1 (r - y), which also leaves y zero on element seams."""
    wl, prob, h, _, scale = case
    tol = TOL64 * scale if dtype == torch.float64 else TOL32
    alpha = 2.0 / 3.0
    for l in range(1, len(h.levels)):
        lv = h.levels[l]
        for s in range(lv.dim):
            x0 = interior_field(lv, 140 + l)
            r = interior_field(lv, 150 + l)
            x = dev(x0, dtype)
            y = torch.zeros(lv.N, dtype=dtype, device="cuda")
            prob.apply(l, x, y)
            prob.line_update(l, s, alpha, dev(r, dtype), y, x)
            ref = h.smoothers[l][s].smooth(x0, r, alpha)
            assert relerr(host(x).reshape(lv.shape), ref) < tol * 10, (l, s)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_restrict_and_prolong(case, dtype):
    wl, prob, h, _, scale = case
    tol = TOL64 * scale if dtype == torch.float64 else TOL32
    for l in range(1, len(h.levels)):
        lf, lc = h.levels[l], h.levels[l - 1]
        r = interior_field(lf, 60 + l)
        x = interior_field(lf, 70 + l)
        rc = torch.zeros(lc.N, dtype=dtype, device="cuda")
        prob.restrict(l, dev(r, dtype), dev(x, dtype), rc)
        ref = h.restrict(l, r - lf.apply(x))
        assert relerr(host(rc).reshape(lc.shape), ref) < tol * 10, l
        e = interior_field(lc, 80 + l)
        xf = dev(x, dtype)
        prob.prolong_add(l, dev(e, dtype), xf)
        ref = x + h.prolong(l, e)
        assert relerr(host(xf).reshape(lf.shape), ref) < tol, l


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_coarse_solve(case, dtype):
    wl, prob, h, _, scale = case
    lv = h.levels[0]
    r = interior_field(lv, 90)
    e = torch.zeros(lv.N, dtype=dtype, device="cuda")
    prob.coarse_solve(dev(r, dtype), e)
    ref = h.coarse_solve(r)
    assert relerr(host(e).reshape(lv.shape), ref) < (1e-11 * scale if dtype == torch.float64 else 1e-4)


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_precondition_gamma_cycle(case, dtype, gamma):
    wl, prob, h, _, scale = case
    fine = h.levels[-1]
    alpha = {"fem": 0.16, "gll": 2.0 / 3.0}.get(h.smoother, 0.5)
    r = interior_field(fine, 100 + gamma)
    z = torch.zeros(fine.N, dtype=dtype, device="cuda")
    prob.precondition(glls.opts(gamma=gamma, alpha=alpha), dev(r, dtype), z)
    ref = h.precondition(r, gamma, alpha)
    tol = 1e-10 * scale if dtype == torch.float64 else 2e-3
    assert relerr(host(z).reshape(fine.shape), ref) < tol


def test_lift(case):
    wl, prob, h, coords, scale = case
    fine = h.levels[-1]
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    f0 = torch.zeros(fine.N, dtype=torch.float64, device="cuda")
    prob.lift(dev(f), dev(g), f0)
    ref, _ = lift(fine, f, g)
    assert relerr(host(f0).reshape(fine.shape), ref) < TOL64 * scale


SOLVE_CASES = [
    ("cfg1_square_sine", inputs.square_sine, "gll", "transpose", 2, 2.0 / 3.0),
    ("2d_6x6_p8", lambda: inputs.random2d((6, 6), 8, amp=0.1, seed=2), "gll", "transpose", 1, 2.0 / 3.0),
    ("2d_6x4_p8_fem", lambda: inputs.random2d((6, 4), 8, amp=0.15, seed=7), "fem", "transpose", 2, 0.16),
    ("2d_single_p8_interp", lambda: inputs.table1_problem3(8), "gll", "interp", 3, 2.0 / 3.0),
    ("2d_3x3_p1", lambda: inputs.random2d((3, 3), 1, amp=0.05, seed=8), "gll", "transpose", 1, 0.5),
    ("2d_single_p2", lambda: inputs.random2d((1, 1), 2, amp=0.0, seed=9), "gll", "transpose", 1, 0.5),
    ("2d_5x4_p7", lambda: inputs.random2d((5, 4), 7, amp=0.1, seed=10), "gll", "transpose", 1, 0.5),
    ("3d_3x3x2_p4", lambda: inputs.random3d((3, 3, 2), 4, amp=0.15, seed=11), "gll", "transpose", 1, 0.5),
    ("3d_2x2x2_p7_fem", lambda: inputs.random3d((2, 2, 2), 7, amp=0.15, seed=12), "fem", "transpose", 1, 0.16),
    ("3d_2x2x3_p6", lambda: inputs.random3d((2, 2, 3), 6, amp=0.1, seed=16), "gll", "transpose", 1, 0.5),
    ("2d_66x66_p8_long_lines", lambda: inputs.random2d((66, 66), 8, amp=0.1, seed=13), "gll", "transpose", 1, 0.5),
    ("3d_3x3x2_p7", lambda: inputs.random3d((3, 3, 2), 7, amp=0.15, seed=20), "gll", "transpose", 1, 2.0 / 3.0),
    ("2d_6x6_p8_band1", lambda: inputs.random2d((6, 6), 8, amp=0.1, seed=2), "gll_band1", "transpose", 1, 0.5),
]


@pytest.mark.parametrize("name,mk,sm,rs,gamma,alpha", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
@pytest.mark.parametrize("use_graph", [2, 1, 0], ids=["device_loop", "graph", "stream"])
def test_solve_fp64_matches_oracle(name, mk, sm, rs, gamma, alpha, use_graph):
    wl = mk()
    prob, h, coords = make(wl, sm, rs)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, gamma=gamma, alpha=alpha, precision=glls.PREC_FP64,
                                 use_graph=use_graph, max_iter=300))
    ref = osolve.solve(wl, gamma=gamma, alpha=alpha, tol=1e-10, maxit=300, hierarchy=h)
    assert relerr(u.reshape(h.levels[-1].shape), ref.u[0]) < 1e-9
    assert abs(st.iterations - ref.iterations[0]) <= 1, (st.iterations, ref.iterations[0])
    assert st.rel_residual <= 1e-10
    prob.close()


@pytest.mark.parametrize("name,mk,sm,rs,gamma,alpha", SOLVE_CASES[:3] + SOLVE_CASES[7:8],
                         ids=[c[0] for c in SOLVE_CASES[:3] + SOLVE_CASES[7:8]])
def test_solve_mixed_reaches_tolerance(name, mk, sm, rs, gamma, alpha):
    """FP32 gamma-cycle inside FP64 FCG reaches the same 1e-10 residual; the
    solution agrees with the FP64 oracle to the tolerance-induced error."""
    wl = mk()
    prob, h, coords = make(wl, sm, rs)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, gamma=gamma, alpha=alpha, precision=glls.PREC_MIXED, max_iter=300))
    ref = osolve.solve(wl, gamma=gamma, alpha=alpha, tol=1e-10, maxit=300, hierarchy=h)
    assert st.rel_residual <= 1e-10
    assert relerr(u.reshape(h.levels[-1].shape), ref.u[0]) < 1e-8
    assert st.iterations <= ref.iterations[0] + 3
    prob.close()


def test_slowly_converging_case_same_solution():
    """Elongated deformed elements (5x3, amp 0.15): about a hundred FCG
    iterations, where rounding order moves the count by a few; the solution
    must still agree."""
    wl = inputs.random2d((5, 3), 8, amp=0.15, seed=2)
    prob, h, coords = make(wl)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=glls.PREC_FP64, max_iter=400))
    ref = osolve.solve(wl, gamma=1, alpha=0.5, tol=1e-10, maxit=400, hierarchy=h)
    assert relerr(u.reshape(h.levels[-1].shape), ref.u[0]) < 1e-9
    assert abs(st.iterations - ref.iterations[0]) <= 0.25 * ref.iterations[0]
    prob.close()


def test_cfg2_full_size_fp64_and_mixed():
    """The benchmark workload (64x64 elements, p = 8, 263,169 nodes) with the
    line blocks at the paper's alpha = 2/3 (9 FCG iterations in the oracle)."""
    wl = inputs.terrain2d()
    prob, h, coords = make(wl, "gll", "transpose")
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    ref = osolve.solve(wl, gamma=1, alpha=2.0 / 3.0, tol=1e-10, maxit=200, hierarchy=h)
    for prec in (glls.PREC_FP64, glls.PREC_MIXED):
        u = np.zeros(prob.N)
        st = prob.solve(u, glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec))
        err = relerr(u.reshape(h.levels[-1].shape), ref.u[0])
        assert err < (1e-9 if prec == glls.PREC_FP64 else 1e-8), (prec, err)
        assert abs(st.iterations - ref.iterations[0]) <= (1 if prec == glls.PREC_FP64 else 3)
    prob.close()


def test_invalid_arguments_are_reported():
    wl = inputs.random2d((2, 2), 3)
    prob, h, coords = make(wl)
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    with pytest.raises(glls.GllsError) as ei:
        prob.apply(7, x, x)
    assert ei.value.status == glls.ERR_INVALID
    with pytest.raises(glls.GllsError):
        prob.line_solve(1, 2, x, x)      # 2-D problem has no axis 2
    with pytest.raises(glls.GllsError):
        prob.solve(np.zeros(prob.N), glls.opts(gamma=0))
    with pytest.raises(glls.GllsError):
        glls.Problem(2, (1, 1), 1, np.zeros((2, 4)))     # single element needs p >= 2
    prob.close()


@pytest.mark.parametrize("name,mk", [("2d_6x6_p8", lambda: inputs.random2d((6, 6), 8, amp=0.1, seed=2)),
                                     ("3d_3x3x2_p7", lambda: inputs.random3d((3, 3, 2), 7, amp=0.15, seed=20)),
                                     ("2d_3x2_p16", lambda: inputs.random2d((3, 2), 16, amp=0.1, seed=15))],
                         ids=lambda v: v if isinstance(v, str) else "")
def test_apply_with_fused_dot_partials(name, mk):
    """The outer iteration's FP64 apply: y = A x and the partials of x.(A x)."""
    wl = mk()
    prob, h, _ = make(wl)
    L = len(h.levels) - 1
    lv = h.levels[L]
    x = interior_field(lv, 7)
    y = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    part = torch.zeros(8192, dtype=torch.float64, device="cuda")
    n = prob.apply_partials(L, dev(x), y, part)
    ref = lv.apply(x)
    assert relerr(host(y).reshape(lv.shape), ref) < TOL64
    dot = float(part[:n].sum())
    assert abs(dot - float(np.vdot(x, ref))) <= 1e-12 * abs(float(np.vdot(x, ref)))
    prob.close()
