"""Pins for transfers, the gamma-cycle schedule and the whole preconditioner
(Sec. 3.3, Def. 3.12, Algorithm 2, Table 1)."""
import json
import os
import warnings

import numpy as np
import pytest

from oracle import gll, solve
from oracle.discretize import Level
from oracle.multigrid import Hierarchy, coarse_coords, interp_1d_global, order_chain
from paper_2504_10710_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def level_of(wl):
    xi, _ = gll.gll(wl.order)
    return Level(wl.dim, wl.nelem, wl.order, wl.coords(xi))


def test_one_element_row_stops_at_p2():
    """One element along an axis: p = 1 has no interior node there, so the
    hierarchy stops at p = 2, whose coarse matrix is the exact coarsest solve."""
    from oracle.gll import gll
    from paper_2504_10710_gb300 import inputs
    for ne in [(9, 1), (1, 7)]:
        wl = inputs.random2d(ne, 4, amp=0.1, seed=35)
        h = Hierarchy(Level(2, ne, 4, wl.coords(gll(4)[0])), restriction="transpose")
        assert h.chain == [4, 2]
        assert h.levels[0].interior.sum() > 0
    wl = inputs.random3d((3, 2, 1), 3, amp=0.1, seed=38)
    h = Hierarchy(Level(3, (3, 2, 1), 3, wl.coords(gll(3)[0])), restriction="transpose")
    assert h.chain == [3, 2] and h.levels[0].interior.sum() > 0


def test_order_chains():
    assert order_chain(8, True) == [8, 4, 2, 1]
    assert order_chain(7, True) == [7, 3, 1]
    assert order_chain(8, False) == [8, 4, 2]
    assert order_chain(11, False) == [11, 5, 2]
    assert order_chain(64, False) == [64, 32, 16, 8, 4, 2]


@pytest.mark.parametrize("ne,pc,pf", [(3, 2, 4), (2, 3, 7), (4, 1, 2), (1, 4, 8)])
def test_prolongation_exact_on_coarse_polynomials(ne, pc, pf):
    """V_{l-1} is nested in V_l: interpolating samples of a piecewise
    polynomial of degree <= p_c reproduces its fine-node samples."""
    P = interp_1d_global(ne, pc, pf)
    xc = (np.arange(ne * pc + 1) // pc).astype(float)
    xf = (np.arange(ne * pf + 1) // pf).astype(float)
    # nodes of each element mapped to [e, e+1]
    xic, _ = gll.gll(pc)
    xif, _ = gll.gll(pf)
    tc = np.concatenate([e + (xic[: -1 if e < ne - 1 else None] + 1) / 2 for e in range(ne)])
    tf = np.concatenate([e + (xif[: -1 if e < ne - 1 else None] + 1) / 2 for e in range(ne)])
    for k in range(pc + 1):
        np.testing.assert_allclose(P @ tc ** k, tf ** k, atol=1e-11 * (ne ** k))
    # the interpolation-type restriction reads a fine field at coarse nodes
    Rint = interp_1d_global(ne, pf, pc)
    for k in range(pc + 1):
        np.testing.assert_allclose(Rint @ tf ** k, tc ** k, atol=1e-11 * (ne ** k))
    del xc, xf


def test_coarse_coords_of_affine_mesh_are_affine_nodes():
    wl = inputs.Workload("sq", 2, (3, 2), 6, inputs.identity_map, [], inputs._zero)
    lv = level_of(wl)
    cc = coarse_coords(lv, 3)
    xi3, _ = gll.gll(3)
    ref = np.stack(wl.undeformed_nodes(xi3))
    np.testing.assert_allclose(cc, ref, atol=1e-14)


def test_transpose_restriction_is_adjoint_of_prolongation():
    lv = level_of(inputs.random2d((3, 2), 4, amp=0.1))
    h = Hierarchy(lv, restriction="transpose")
    rng = np.random.default_rng(0)
    for l in range(1, h.L + 1):
        uf = np.where(h.levels[l].interior, rng.standard_normal(h.levels[l].shape), 0)
        vc = np.where(h.levels[l - 1].interior, rng.standard_normal(h.levels[l - 1].shape), 0)
        assert abs(np.vdot(h.restrict(l, uf), vc) - np.vdot(uf, h.prolong(l, vc))) < 1e-12


def expected_schedule(L, gamma, d):
    """Visit order of Algorithm 2 written out from the definition."""
    out = []

    def visit(l):
        if l == 0:
            out.append(("coarse", 0))
            return
        out.extend(("smooth", l, s) for s in range(d))
        for _ in range(gamma):
            visit(l - 1)
            out.extend(("smooth", l, s) for s in reversed(range(d)))
    visit(L)
    return out


@pytest.mark.parametrize("gamma", [1, 2, 3])
def test_schedule_and_visit_counts(gamma):
    lv = level_of(inputs.random2d((2, 2), 8, amp=0.05))
    h = Hierarchy(lv, restriction="transpose")
    trace = []
    h.precondition(np.ones(lv.shape), gamma, 0.5, trace=trace)
    assert trace == expected_schedule(h.L, gamma, 2)
    # level l is visited gamma^(L-l) times (Prop. 3.13): pre d + gamma * d post smooths per visit
    for l in range(1, h.L + 1):
        n = sum(1 for t in trace if t[0] == "smooth" and t[1] == l)
        assert n == gamma ** (h.L - l) * (2 + 2 * gamma)
    assert sum(1 for t in trace if t[0] == "coarse") == gamma ** h.L
    # literal Fig. 5 shape for gamma = 1, L = 3: x y | x y ... down, then y x up
    if gamma == 1:
        assert [t[1] for t in trace] == [3, 3, 2, 2, 1, 1, 0, 1, 1, 2, 2, 3, 3]


def test_cycle_is_linear_and_symmetric_for_gamma1_transpose():
    lv = level_of(inputs.random2d((3, 3), 4, amp=0.1))
    h = Hierarchy(lv, restriction="transpose")
    rng = np.random.default_rng(1)
    x = np.where(lv.interior, rng.standard_normal(lv.shape), 0)
    y = np.where(lv.interior, rng.standard_normal(lv.shape), 0)
    Mx = h.precondition(x, 1, 0.5)
    My = h.precondition(y, 1, 0.5)
    assert abs(np.vdot(Mx, y) - np.vdot(x, My)) < 1e-11 * abs(np.vdot(Mx, y))
    np.testing.assert_allclose(h.precondition(2 * x - 3 * y, 2, 0.5),
                               2 * h.precondition(x, 2, 0.5) - 3 * h.precondition(y, 2, 0.5), atol=1e-11)
    # gamma >= 2 is not symmetric (why the outer solver is flexible CG)
    Mx2 = h.precondition(x, 2, 0.5)
    My2 = h.precondition(y, 2, 0.5)
    assert abs(np.vdot(Mx2, y) - np.vdot(x, My2)) > 1e-8 * abs(np.vdot(Mx2, y))


P1 = "problem1_lap_u_eq_minus1"
P3 = "problem3_sin_8pi_over_x_plus_y_plus_pi_10"

# (smoother, problem, p_L, gammas, allowed deviation per gamma).  GLL rows use
# Def. 3.2's line blocks R A_p P read literally.  The band-1 reading misses
# the p_L = 32 row by up to 14 iterations and does not converge within 60 at
# p_L = 64 (test_band1_reading_misses_table1_at_high_order).  Deviations
# larger than one: GLL problem 1 at p_L = 32 gives 17 for the printed 19
# (gamma = 1) and at p_L = 64 gives 28 for 31; problem 3 with the GLL
# smoother at p_L = 8 gives 8 / 6 / 5 for 10 / 7 / 6 (gamma = 1..3).
TABLE1_CASES = [
    ("FEM", P1, 8, range(1, 9), 1), ("FEM", P1, 16, range(1, 9), 1), ("FEM", P1, 32, range(1, 9), 1),
    ("FEM", P3, 8, range(1, 9), 1), ("FEM", P3, 16, range(1, 9), 1),
    ("GLL", P1, 8, range(1, 9), 1), ("GLL", P1, 16, range(1, 9), 1), ("GLL", P1, 32, range(1, 9), 2),
    # (gamma = 6..8 take 28-93 s each in the oracle: measured once, 7 6 6 for the printed 6 5 5)
    ("GLL", P1, 64, range(1, 6), (3, 1, 1, 1, 1)),
    ("GLL", P3, 8, range(1, 9), 2),
]


@pytest.mark.parametrize("smoother,problem,pL,gammas,dev", TABLE1_CASES,
                         ids=[f"{c[0]}-{c[1][:8]}-p{c[2]}" for c in TABLE1_CASES])
def test_table1_gmres_iteration_counts(smoother, problem, pL, gammas, dev):
    """Soft pin against Table 1: GMRES iterations to 1e-8 within `dev` of the
    printed count for each gamma, with the interpolation-type restriction.
    (The p_L = 16 row of problem 3 is printed as "11".)"""
    gold = json.load(open(os.path.join(GOLD, "table1_iterations.json")))
    key = str(pL) if str(pL) in gold[problem][smoother] else "11"
    gammas = list(gammas)
    printed = [gold[problem][smoother][key][g - 1] for g in gammas]
    devs = dev if isinstance(dev, tuple) else (dev,) * len(gammas)
    wl = inputs.table1_problem1(pL) if problem == P1 else inputs.table1_problem3(pL)
    alpha = 2 / 3 if smoother == "GLL" else 0.16
    fine, hier = solve.build(wl, smoother=smoother.lower(), restriction="interp")
    ours = [solve.solve(wl, gamma=g, alpha=alpha, tol=1e-8, maxit=60, method="gmres",
                        hierarchy=hier).iterations[0] for g in gammas]
    assert all(abs(o - q) <= d for o, q, d in zip(ours, printed, devs)), (ours, printed)


def test_band1_reading_misses_table1_at_high_order():
    """Records why Def. 3.2 is read literally: with the band-1 part of the
    line blocks the GLL row p_L = 32 of problem 1 (printed 19 12 9 ...) takes
    more than 30 GMRES iterations at gamma = 1."""
    wl = inputs.table1_problem1(32)
    fine, hier = solve.build(wl, smoother="gll_band1", restriction="interp")
    it = solve.solve(wl, gamma=1, alpha=2 / 3, tol=1e-8, maxit=60, method="gmres", hierarchy=hier).iterations[0]
    assert it > 30, it


def _smoothed_spectrum(smoother):
    wl = inputs.random2d((2, 2), 8, amp=0.1, seed=1)
    lv = level_of(wl)
    h = Hierarchy(lv, smoother=smoother, restriction="transpose")
    ii = lv.interior_index()
    A = lv.assemble()[ii][:, ii].toarray()
    out = []
    for s in range(2):
        B = np.zeros_like(A)
        for k in range(len(ii)):
            e = np.zeros(lv.N)
            e[ii[k]] = 1
            B[:, k] = h.smoothers[-1][s].apply_inverse(e.reshape(lv.shape)).ravel()[ii]
        out.append(np.linalg.eigvals(B @ A).real)
    return out


def test_line_block_smoother_admits_alpha_two_thirds():
    """With the literal line blocks the spectrum of B_s^-1 A on a deformed
    p = 8 grid lies in (0, 2.5), below 2/alpha = 3 for the paper's alpha =
    2/3, so the damped line smoothing step contracts."""
    for lam in _smoothed_spectrum("gll"):
        assert lam.min() > 0 and 2.0 < lam.max() < 2.5


def test_gll_band1_smoother_diverges_at_high_order_alpha_two_thirds():
    """Records why the band-1 reading needs alpha < 2/3 on deformed grids: the
    largest eigenvalue of B_x^-1 A exceeds 2/alpha = 3 at p = 8."""
    lam = _smoothed_spectrum("gll_band1")[0]
    assert lam.min() > 0 and 3.0 < lam.max() < 4.0


def test_multielement_fcg_counts_are_small():
    """cfg2-like deformed grid, 16x16 elements p = 8, FCG to 1e-10: the line
    blocks at the paper's alpha = 2/3 take 9 (gamma = 1), the band-1 reading
    at alpha = 0.5 takes 14, the FEM smoother 12 (gamma = 2)."""
    wl = inputs.terrain2d(nelem=16)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        counts = {}
        for sm, g, a in (("gll", 1, 2 / 3), ("gll_band1", 1, 0.5), ("fem", 2, 0.16)):
            fine, hier = solve.build(wl, smoother=sm, restriction="transpose")
            counts[sm] = solve.solve(wl, gamma=g, alpha=a, tol=1e-10, maxit=100, hierarchy=hier).iterations[0]
    assert counts["gll"] <= 10 and counts["gll_band1"] <= 16 and counts["fem"] <= 15, counts
