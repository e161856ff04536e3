"""The float-float outer apply (q = A p with the p.(A p) partials, each value a
pair of FP32 numbers) against the oracle's FP64 operator, its refusals, and
the mixed-precision solve that runs it: the true residual f - A u, computed by
the oracle, stays at the solver tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.discretize import Level, lift  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402

# about 48 significant bits: a contraction of 2 (p + 1) terms rounds near
# 2^-44 of its largest term, so the element sums land well inside 1e-12 of the
# largest output; (p / 8)^2 scales it with the derivative entries as the FP64
# parity tests do
TOL_FF = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    ("2d_6x6_p8", lambda: inputs.random2d((6, 6), 8, amp=0.1, seed=2)),
    ("2d_7x5_p2", lambda: inputs.random2d((7, 5), 2, amp=0.1, seed=31)),
    ("2d_5x4_p5", lambda: inputs.random2d((5, 4), 5, amp=0.15, seed=32)),
    ("2d_4x3_p12", lambda: inputs.random2d((4, 3), 12, amp=0.1, seed=33)),
    ("2d_3x2_p16", lambda: inputs.random2d((3, 2), 16, amp=0.1, seed=15)),
    ("2d_single_p9", lambda: inputs.table1_problem3(9)),
    # the bench grid (263,169 nodes): its sums' terms exceed the output by
    # about 1e3, and the FP64 apply itself is 2e-12 from the oracle there
    ("2d_64x64_p8_bench", lambda: inputs.terrain2d(), 4),
    # 3-D: the even-odd line kernel, odd and even orders, ragged element counts
    ("3d_3x3x2_p7", lambda: inputs.random3d((3, 3, 2), 7, amp=0.15, seed=20)),
    ("3d_2x2x2_p8", lambda: inputs.random3d((2, 2, 2), 8, amp=0.1, seed=36)),
    ("3d_3x2x4_p4", lambda: inputs.random3d((3, 2, 4), 4, amp=0.1, seed=37)),
    ("3d_5x3x2_p2", lambda: inputs.random3d((5, 3, 2), 2, amp=0.1, seed=38)),
    ("3d_2x3x2_p5", lambda: inputs.random3d((2, 3, 2), 5, amp=0.15, seed=39)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_ff_apply_and_partials_match_oracle(case):
    wl = case[1]()
    prob, coords = glls.problem_for(wl)
    lv = Level(wl.dim, wl.nelem, wl.order, coords)
    rng = np.random.default_rng(3)
    x = np.where(lv.interior, rng.standard_normal(lv.shape), 0.0)
    L = prob.levels - 1
    xd = torch.tensor(x.ravel(), dtype=torch.float64, device="cuda")
    part = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    y = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    n = prob.apply_partials(L, xd, y, part, ff=True)
    y64 = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    part64 = torch.zeros_like(part)
    n64 = prob.apply_partials(L, xd, y64, part64)
    torch.cuda.synchronize()
    if wl.dim == 2:
        assert n == n64          # the same CTAs as the FP64 node-per-thread kernel
    ref = lv.apply(x)
    scale = max(1.0, (wl.order / 8.0) ** 2) * (case[2] if len(case) > 2 else 1)
    got = y.cpu().numpy().reshape(lv.shape)
    assert _rel(got, ref) < TOL_FF * scale
    assert _rel(got, y64.cpu().numpy().reshape(lv.shape)) < TOL_FF * scale
    dot, rdot = float(part[:n].sum()), float(np.vdot(x, ref))
    assert abs(dot - rdot) <= 1e-12 * scale * abs(rdot)
    # the rounding is that of about 48 bits, not of FP32 (which would be ~1e-7)
    assert _rel(got, ref) < 2e-11
    prob.close()


@pytest.mark.parametrize("scale", [1e-20, 1e-8, 1e8, 1e25], ids=lambda v: f"x{v:g}")
@pytest.mark.parametrize("mk", [lambda: inputs.random2d((5, 4), 6, amp=0.1, seed=44),
                                lambda: inputs.random3d((3, 2, 2), 7, amp=0.1, seed=45)], ids=["2d", "3d"])
def test_ff_apply_scaled_inputs(mk, scale):
    """The conversions between FP64 and float pairs across the FP32 exponent
    range: p scaled by 1e-20 .. 1e25 gives A p scaled the same, to the same
    relative accuracy."""
    wl = mk()
    prob, coords = glls.problem_for(wl)
    lv = Level(wl.dim, wl.nelem, wl.order, coords)
    rng = np.random.default_rng(9)
    x = np.where(lv.interior, rng.standard_normal(lv.shape), 0.0) * scale
    L = prob.levels - 1
    part = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    y = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    n = prob.apply_partials(L, torch.tensor(x.ravel(), dtype=torch.float64, device="cuda"), y, part, ff=True)
    torch.cuda.synchronize()
    ref = lv.apply(x)
    assert _rel(y.cpu().numpy().reshape(lv.shape), ref) < TOL_FF
    rdot = float(np.vdot(x, ref))
    assert abs(float(part[:n].sum()) - rdot) <= 1e-12 * abs(rdot)
    prob.close()


def test_ff_apply_refusals():
    part = torch.zeros(1 << 12, dtype=torch.float64, device="cuda")
    # a coarse level (the float-float factors are kept for the finest level only)
    wl = inputs.random2d((4, 4), 4, amp=0.1, seed=34)
    prob, _ = glls.problem_for(wl)
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    with pytest.raises(glls.GllsError) as ei:
        prob.apply_partials(prob.levels - 2, x, x.clone(), part, ff=True)
    assert ei.value.status == glls.ERR_INVALID
    prob.close()
    # an order above the float-float kernels' range, and coloured summation
    for w, kw in ((inputs.random2d((3, 3), 17, amp=0.05, seed=35), {}),
                  (wl, {"summation": glls.SUM_COLORED})):
        prob, _ = glls.problem_for(w, **kw)
        x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
        with pytest.raises(glls.GllsError) as ei:
            prob.apply_partials(prob.levels - 1, x, x.clone(), part, ff=True)
        assert ei.value.status == glls.ERR_INVALID
        prob.close()


@pytest.mark.parametrize("tol", [1e-10, 1e-12], ids=["tol1e-10", "tol1e-12"])
@pytest.mark.parametrize("mk", [inputs.terrain2d, lambda: inputs.random3d((6, 5, 4), 7, amp=0.1, seed=40)],
                         ids=["2d_64x64_p8_bench", "3d_6x5x4_p7"])
def test_mixed_solve_true_residual_at_tolerance(tol, mk):
    """Mixed precision with the float-float outer apply (line blocks,
    alpha = 2/3): the recurrence residual the solver reports and the true
    residual of the returned u (oracle, FP64) agree, both at the tolerance."""
    wl = mk()
    prob, coords = glls.problem_for(wl)
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    prob.set_rhs(f)
    prob.set_dirichlet(g)
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=tol, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED))
    assert st.status == glls.OK and st.rel_residual <= tol
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    f0, v = lift(fine, f, g)
    w = u.reshape(fine.shape) - v
    true = np.linalg.norm(f0 - fine.apply(w)) / np.linalg.norm(f0)
    assert true <= 1.5 * tol, (true, st.rel_residual)
    prob.close()


def test_worklist_batch_with_ff_apply_equals_single_solves():
    """Work-list batch in mixed precision (its outer apply in float-float, as
    the single solves'): each problem gets its single-solve result."""
    ws = [inputs.random2d((9, 7), 6, amp=0.1, seed=41), inputs.random2d((12, 10), 8, amp=0.1, seed=42),
          inputs.random2d((5, 6), 5, amp=0.1, seed=43)]
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    probs, single, its = [], [], []
    for w in ws:
        p, coords = glls.problem_for(w)
        p.set_rhs(w.sample_rhs(coords)[0])
        p.set_dirichlet(w.sample_dirichlet(coords))
        u = np.zeros(p.N)
        its.append(p.solve(u, o).iterations)
        single.append(u)
        probs.append(p)
    outs = [np.zeros(p.N) for p in probs]
    stats = glls.solve_batch(probs, outs, o, worklist=True)
    for u, ub, s, k in zip(single, outs, stats, its):
        assert _rel(ub, u) < 1e-8 and abs(s.iterations - k) <= 1 and s.status == glls.OK
    for p in probs:
        p.close()
