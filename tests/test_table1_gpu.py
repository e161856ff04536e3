"""Table 1 of the paper through the CUDA path: right-preconditioned GMRES
(the paper's outer solver) with the gamma-cycle on a single GLL element,
residual reduction 1e-8, interpolation-type restriction.  Iteration counts
equal the oracle's GMRES counts (within one) and the printed Table 1 values
(within one; two for the GLL line blocks at p_L = 32) for every gamma = 1..8;
the GMRES solution equals the oracle's."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solve as osolve  # noqa: E402
from oracle.discretize import Level  # noqa: E402
from oracle.multigrid import Hierarchy  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [("FEM", "problem1_lap_u_eq_minus1", 8), ("FEM", "problem1_lap_u_eq_minus1", 16),
         ("FEM", "problem3_sin_8pi_over_x_plus_y_plus_pi_10", 8),
         ("FEM", "problem3_sin_8pi_over_x_plus_y_plus_pi_10", 16),
         ("GLL", "problem1_lap_u_eq_minus1", 8), ("GLL", "problem1_lap_u_eq_minus1", 16),
         ("GLL", "problem1_lap_u_eq_minus1", 32)]
# largest deviation from the printed counts (the oracle's own, see
# tests/test_oracle_multigrid.py): GLL p_L = 32 gives 17 for the printed 19 at gamma = 1
PRINTED_DEV = {("GLL", 32): 2}


@pytest.mark.parametrize("smoother,problem,pL", CASES, ids=[f"{a}-{b[:8]}-p{c}" for a, b, c in CASES])
def test_table1_gmres_counts_on_gpu(smoother, problem, pL):
    gold = json.load(open(os.path.join(GOLD, "table1_iterations.json")))
    key = str(pL) if str(pL) in gold[problem][smoother] else "11"
    printed = gold[problem][smoother][key]
    wl = inputs.table1_problem1(pL) if problem.startswith("problem1") else inputs.table1_problem3(pL)
    alpha = 2 / 3 if smoother == "GLL" else 0.16
    sm = glls.SMOOTHER_GLL if smoother == "GLL" else glls.SMOOTHER_FEM
    prob, coords = glls.problem_for(wl, sm, glls.RESTRICT_INTERP)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    hier = Hierarchy(fine, smoother=smoother.lower(), restriction="interp")
    gpu, ora = [], []
    for g in range(1, 9):
        u = np.zeros(prob.N)
        st = prob.solve(u, glls.opts(tol=1e-8, gamma=g, alpha=alpha, precision=glls.PREC_FP64,
                                     krylov=glls.KRYLOV_GMRES, max_iter=60))
        ref = osolve.solve(wl, gamma=g, alpha=alpha, tol=1e-8, maxit=60, method="gmres", hierarchy=hier)
        gpu.append(st.iterations)
        ora.append(ref.iterations[0])
        np.testing.assert_allclose(u, ref.u[0].ravel(), atol=1e-9 * np.abs(ref.u[0]).max())
    assert all(abs(a - b) <= 1 for a, b in zip(gpu, ora)), (gpu, ora)
    dev = PRINTED_DEV.get((smoother, pL), 1)
    assert all(abs(a - b) <= dev for a, b in zip(gpu, printed)), (gpu, printed)
    prob.close()


def test_gmres_multielement_mixed_and_fp64():
    wl = inputs.random2d((6, 6), 8, amp=0.1, seed=2)
    prob, coords = glls.problem_for(wl)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    hier = Hierarchy(fine, restriction="transpose")
    ref = osolve.solve(wl, gamma=1, alpha=0.5, tol=1e-10, maxit=100, method="gmres", hierarchy=hier)
    for prec in (glls.PREC_FP64, glls.PREC_MIXED):
        u = np.zeros(prob.N)
        st = prob.solve(u, glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=prec, krylov=glls.KRYLOV_GMRES,
                                     max_iter=100))
        assert st.rel_residual <= 1e-10
        assert np.abs(u - ref.u[0].ravel()).max() <= 1e-8 * np.abs(ref.u[0]).max()
        assert abs(st.iterations - ref.iterations[0]) <= (1 if prec == glls.PREC_FP64 else 3)
    prob.close()
