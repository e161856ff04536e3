"""Block cyclic reduction of the coarsest level (Thm. 3.8 with m > 1, Cor.
3.9) on the GPU: every depth against the oracle's direct coarse solve
(Cholesky of the assembled A_0), whole solves with it, and the full-size
64 x 64, p = 8 workload.  Tolerances as for the dense coarse solve: 1e-11
(FP64) and 1e-4 (FP32) relative to the largest entry."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import blockcr  # noqa: E402
from oracle.discretize import Level  # noqa: E402
from oracle.multigrid import Hierarchy, coarse_coords  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


GRIDS = [("2d_9x7_p2", lambda: inputs.random2d((9, 7), 2, amp=0.1, seed=41)),      # 6 blocks of 8
         ("2d_16x16_p4", lambda: inputs.random2d((16, 16), 4, amp=0.1, seed=42)),  # 15 blocks of 15
         ("2d_5x13_p3", lambda: inputs.random2d((5, 13), 3, amp=0.15, seed=43)),   # 12 blocks of 4
         ("3d_4x3x5_p2", lambda: inputs.random3d((4, 3, 5), 2, amp=0.1, seed=44)),  # 4 planes of 6
         ("3d_3x3x8_p3", lambda: inputs.random3d((3, 3, 8), 3, amp=0.1, seed=45))]  # 7 planes of 4


def _max_levels(nb):
    k = 0
    while (2 << k) <= nb:
        k += 1
    return k


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("grid", GRIDS, ids=[g[0] for g in GRIDS])
def test_coarse_solve_every_depth(grid):
    wl = grid[1]()
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    hier = Hierarchy(Level(wl.dim, wl.nelem, wl.order, coords), restriction="transpose")
    lv = hier.levels[0]
    nb = lv.shape[0] - 2
    m = int(np.prod([n - 2 for n in lv.shape[1:]]))
    r = np.where(lv.interior, inputs.random_field(lv.shape, 7), 0.0)
    ref = hier.coarse_solve(r)
    # the oracle's block CR at full depth reaches the same solution
    ii = lv.interior_index()
    A, L, U, nb_o, m_o = blockcr.grid_blocks(lv.assemble()[ii][:, ii].toarray(), tuple(n - 2 for n in lv.shape[::-1]))
    assert (nb_o, m_o) == (nb, m)
    assert _relerr(blockcr.block_cr_solve(A, L, U, r.ravel()[ii]), ref.ravel()[ii]) < 1e-11
    for k in range(0, _max_levels(nb) + 1):
        solver = glls.COARSE_DENSE if k == 0 else glls.COARSE_BLOCK_CR
        prob = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=solver, coarse_cr_levels=k)
        assert prob.info.coarse_cr_levels == k
        assert prob.info.coarse_dense_unknowns == (nb >> k) * m
        for dtype, tol in ((torch.float64, 1e-11), (torch.float32, 1e-4)):
            e = torch.zeros(lv.N, dtype=dtype, device="cuda")
            prob.coarse_solve(torch.tensor(r.ravel(), dtype=dtype, device="cuda"), e)
            torch.cuda.synchronize()
            assert _relerr(e.double().cpu().numpy().reshape(lv.shape), ref) < tol, (k, dtype)
        prob.close()


def test_block_cr_levels_are_clamped_and_auto_is_valid():
    wl = inputs.random2d((9, 7), 2, amp=0.1, seed=41)       # 6 blocks: at most 2 levels
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    p = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=glls.COARSE_BLOCK_CR, coarse_cr_levels=9)
    assert p.info.coarse_cr_levels == 2
    p.close()
    p = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=glls.COARSE_BLOCK_CR)
    assert 1 <= p.info.coarse_cr_levels <= 2
    p.close()
    p = glls.Problem(wl.dim, wl.nelem, wl.order, coords)
    assert 0 <= p.info.coarse_cr_levels <= 2
    p.close()
    with pytest.raises(glls.GllsError):
        glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=7)


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
def test_solves_with_block_cr_equal_dense(prec):
    wl = inputs.random2d((12, 10), 6, amp=0.1, seed=46)
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=prec)
    sols, its = [], []
    for solver, k in ((glls.COARSE_DENSE, 0), (glls.COARSE_BLOCK_CR, 1), (glls.COARSE_BLOCK_CR, 3)):
        prob = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=solver, coarse_cr_levels=k)
        prob.set_rhs(f)
        prob.set_dirichlet(g)
        u = np.zeros(prob.N)
        st = prob.solve(u, o)
        assert st.rel_residual <= 1e-10
        sols.append(u)
        its.append(st.iterations)
        prob.close()
    for u, k in zip(sols[1:], its[1:]):
        assert _relerr(u, sols[0]) < 1e-9
        assert abs(k - its[0]) <= 1


def test_full_size_coarse_level_64x64_p8():
    """The 64 x 64, p = 8 workload: coarsest level p = 1 with 63 blocks of 63
    unknowns; the automatic depth and every explicit depth agree with the
    oracle's direct coarse solve."""
    wl = inputs.terrain2d()
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    hier = Hierarchy(fine, restriction="transpose")
    lv = hier.levels[0]
    r = np.where(lv.interior, inputs.random_field(lv.shape, 8), 0.0)
    ref = hier.coarse_solve(r)
    for solver, k in ((glls.COARSE_AUTO, 0), (glls.COARSE_BLOCK_CR, 1), (glls.COARSE_BLOCK_CR, 2),
                      (glls.COARSE_BLOCK_CR, 5)):
        prob = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=solver, coarse_cr_levels=k)
        for dtype, tol in ((torch.float64, 1e-11), (torch.float32, 1e-4)):
            e = torch.zeros(lv.N, dtype=dtype, device="cuda")
            prob.coarse_solve(torch.tensor(r.ravel(), dtype=dtype, device="cuda"), e)
            torch.cuda.synchronize()
            assert _relerr(e.double().cpu().numpy().reshape(lv.shape), ref) < tol, (solver, k, dtype)
        prob.close()


@pytest.mark.parametrize("k", [0, 1, 3])
def test_estimate_bytes_tracks_block_cr_allocation(k):
    wl = inputs.random2d((16, 16), 4, amp=0.1, seed=42)
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    solver = glls.COARSE_DENSE if k == 0 else glls.COARSE_BLOCK_CR
    prob = glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=solver, coarse_cr_levels=k)
    est = glls.estimate_bytes(wl.dim, wl.nelem, wl.order, coords, coarse_solver=solver, coarse_cr_levels=k)
    actual = prob.info.device_bytes
    assert 0.8 * actual <= est <= 1.25 * actual, (est, actual)
    prob.close()


def _coarse_residual(wl, prob, lv, seed):
    """||r - A_0 e|| / ||r|| for e = the library's coarse solve of a random r,
    with A_0 applied by the oracle's matrix-free operator."""
    r = np.where(lv.interior, inputs.random_field(lv.shape, seed), 0.0)
    out = []
    for dtype in (torch.float64, torch.float32):
        e = torch.zeros(lv.N, dtype=dtype, device="cuda")
        prob.coarse_solve(torch.tensor(r.ravel(), dtype=dtype, device="cuda"), e)
        torch.cuda.synchronize()
        ev = e.double().cpu().numpy().reshape(lv.shape)
        out.append(np.linalg.norm(r - lv.apply(ev)) / np.linalg.norm(r))
    return out


def test_coarsest_level_above_the_dense_limit_takes_block_cr():
    """27^3 elements put 26^3 = 17,576 unknowns on the p = 1 level, above the
    16,384 of the dense inverse: AUTO takes block CR over the 26 planes, the
    coarse solve inverts A_0 (residual check with the oracle's operator), the
    whole solve converges, and the dense solver alone is refused."""
    wl = inputs.random3d((27, 27, 27), 2, amp=0.1, seed=47)
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    with pytest.raises(glls.GllsError) as err:
        glls.Problem(wl.dim, wl.nelem, wl.order, coords, coarse_solver=glls.COARSE_DENSE)
    assert err.value.status == glls.ERR_INVALID
    prob = glls.Problem(wl.dim, wl.nelem, wl.order, coords)
    assert prob.info.coarse_cr_levels >= 1 and prob.info.coarse_unknowns == 26 ** 3
    fine = Level(wl.dim, wl.nelem, wl.order, coords)
    lv0 = Level(3, wl.nelem, 1, coarse_coords(fine, 1))
    r64, r32 = _coarse_residual(wl, prob, lv0, 9)
    assert r64 < 1e-10 and r32 < 1e-4, (r64, r32)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED))
    assert st.status == glls.OK and st.rel_residual <= 1e-10
    prob.close()


def test_largest_serving_coarsest_level_32_cubed():
    """The largest 3-D serving mesh, 32^3 elements, has 31^3 = 29,791
    unknowns on its p = 1 level.  At p = 1 that level is the whole problem:
    block CR over 31 planes of 961 unknowns is its exact inverse, so the
    preconditioned solve converges in one iteration."""
    wl = inputs.random3d((32, 32, 32), 1, amp=0.15, seed=48)
    xi, _ = glls.gll(1)
    coords = wl.coords(xi)
    prob = glls.Problem(wl.dim, wl.nelem, 1, coords)
    assert prob.info.coarse_unknowns == 31 ** 3 and prob.info.coarse_cr_levels >= 1
    lv = Level(3, wl.nelem, 1, coords)
    r64, r32 = _coarse_residual(wl, prob, lv, 10)
    assert r64 < 1e-10 and r32 < 1e-4, (r64, r32)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_FP64))
    assert st.status == glls.OK and st.iterations <= 2
    prob.close()
