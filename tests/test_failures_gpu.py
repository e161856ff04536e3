"""Failure paths of the C ABI, each made on the host: bad data (a NaN in f),
an iteration cap, a folded mesh, an injected device-allocation failure, and
the caller's current device restored by every entry point.  Nothing here
faults or hangs the GPU: every failure is a status the library reports."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_10710_gb300 import glls, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _problem(wl=None):
    wl = wl or inputs.random2d((5, 4), 6, amp=0.1, seed=51)
    prob, coords = glls.problem_for(wl)
    prob.set_rhs(wl.sample_rhs(coords)[0])
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    return wl, prob, coords


@pytest.mark.parametrize("use_graph", [2, 1, 0], ids=["device_loop", "graph", "stream"])
@pytest.mark.parametrize("krylov", [glls.KRYLOV_FCG, glls.KRYLOV_GMRES], ids=["fcg", "gmres"])
def test_nan_in_rhs_reports_breakdown(use_graph, krylov):
    wl, prob, coords = _problem()
    f = np.array(wl.sample_rhs(coords)[0], dtype=np.float64).ravel()
    nx = prob.level_shape(prob.levels - 1)[-1]
    f[10 * nx + 10] = np.nan             # an interior node (boundary values of f are not used)
    prob.set_rhs(f)
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_MIXED, use_graph=use_graph, krylov=krylov),
                    raise_on_error=False)
    assert st.status == glls.ERR_BREAKDOWN, st.status
    # the problem stays usable: clean data solves again
    prob.set_rhs(wl.sample_rhs(coords)[0])
    st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_MIXED, use_graph=use_graph, krylov=krylov))
    assert st.status == glls.OK and np.isfinite(u).all()
    prob.close()


@pytest.mark.parametrize("use_graph", [2, 1, 0], ids=["device_loop", "graph", "stream"])
def test_iteration_cap_reports_not_converged_with_last_iterate(use_graph):
    wl, prob, coords = _problem()
    full = np.zeros(prob.N)
    st_full = prob.solve(full, glls.opts(tol=1e-10, precision=glls.PREC_FP64, use_graph=use_graph))
    assert st_full.iterations > 3
    u = np.full(prob.N, np.nan)
    st = prob.solve(u, glls.opts(tol=1e-10, max_iter=2, precision=glls.PREC_FP64, use_graph=use_graph),
                    raise_on_error=False)
    assert st.status == glls.ERR_NOT_CONVERGED
    assert st.iterations == 2 and 1e-10 < st.rel_residual < 1.0
    # the last iterate is written: finite, with the Dirichlet data on the boundary,
    # closer to the converged solution than the lifting alone
    assert np.isfinite(u).all()
    g = np.asarray(wl.sample_dirichlet(coords), dtype=np.float64)
    shape = prob.level_shape(prob.levels - 1)
    bd = np.ones(shape, dtype=bool)
    bd[tuple(slice(1, -1) for _ in shape)] = False
    np.testing.assert_array_equal(u.reshape(shape)[bd], g.reshape(shape)[bd])
    lift_only = np.where(bd, g.reshape(shape), 0.0).ravel()
    assert np.abs(u - full).max() < np.abs(lift_only - full).max()
    prob.close()


def test_folded_mesh_is_refused_at_setup():
    """Two node columns of an element swapped: the isoparametric map folds
    and its Jacobian changes sign, so set-up refuses the mesh."""
    wl = inputs.random2d((3, 3), 4, amp=0.05, seed=52)
    xi, _ = glls.gll(wl.order)
    coords = np.array(wl.coords(xi), dtype=np.float64).reshape(2, 13, 13)
    coords[0][:, [1, 3]] = coords[0][:, [3, 1]]
    with pytest.raises(glls.GllsError) as ei:
        glls.Problem(2, wl.nelem, wl.order, coords.reshape(2, -1))
    assert ei.value.status == glls.ERR_BREAKDOWN
    assert "jacobian" in str(ei.value).lower()


def test_injected_allocation_failure_reports_oom_and_frees():
    wl = inputs.random2d((8, 8), 6, amp=0.1, seed=53)
    xi, _ = glls.gll(wl.order)
    coords = np.asarray(wl.coords(xi))
    glls.Problem(2, wl.nelem, wl.order, coords).close()     # warm-up (kernel attributes, context)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n in (0, 3, 20, 60):
        glls.lib().glls_debug_fail_alloc_after(n)
        try:
            with pytest.raises(glls.GllsError) as ei:
                glls.Problem(2, wl.nelem, wl.order, coords)
        finally:
            glls.lib().glls_debug_fail_alloc_after(-1)
        assert ei.value.status == glls.ERR_OOM, (n, ei.value)
    torch.cuda.synchronize()
    # what the failed set-ups allocated was released (allow allocator slack)
    assert free0 - torch.cuda.mem_get_info()[0] < 16 << 20
    prob = glls.Problem(2, wl.nelem, wl.order, coords)
    # a clone that cannot allocate fails the same way and leaves the original usable
    glls.lib().glls_debug_fail_alloc_after(2)
    try:
        with pytest.raises(glls.GllsError) as ei:
            prob.clone()
    finally:
        glls.lib().glls_debug_fail_alloc_after(-1)
    assert ei.value.status == glls.ERR_OOM
    f = wl.sample_rhs(coords)[0]
    prob.set_rhs(f)
    prob.set_dirichlet(wl.sample_dirichlet(coords))
    u = np.zeros(prob.N)
    assert prob.solve(u, glls.opts(tol=1e-10)).status == glls.OK
    prob.close()


def test_entry_points_restore_the_callers_device():
    """The library makes the problem's device current for a call and restores
    the caller's current device afterwards (checked here on device 0: the
    caller's device is what cudaGetDevice reports after each call)."""
    wl, prob, coords = _problem()
    dev_before = torch.cuda.current_device()
    u = np.zeros(prob.N)
    prob.solve(u, glls.opts(tol=1e-10))
    x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    prob.apply(prob.levels - 1, x, y)
    c = prob.clone()
    c.close()
    assert torch.cuda.current_device() == dev_before
    prob.close()


@pytest.mark.parametrize("scale", [1e40, 1e-50], ids=["x1e40", "x1e-50"])
def test_mixed_solve_outside_fp32_range_reports_breakdown(scale):
    """Data far outside the FP32 exponent range: the mixed solve (FP32 cycle,
    float-float outer apply) reports a breakdown instead of a wrong answer;
    the same problem then solves the same data in FP64, and ordinary data in
    mixed precision (the breakdown's Inf/NaN do not stay in its work
    vectors)."""
    wl, prob, coords = _problem()
    f = np.asarray(wl.sample_rhs(coords)[0], dtype=np.float64)
    prob.set_rhs(f * scale)
    prob.set_dirichlet(np.zeros(prob.N))
    u = np.zeros(prob.N)
    st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_MIXED), raise_on_error=False)
    assert st.status == glls.ERR_BREAKDOWN, st.status
    st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_FP64))
    assert st.status == glls.OK and np.isfinite(u).all()
    prob.set_rhs(f)
    for use_graph in (2, 0):
        st = prob.solve(u, glls.opts(tol=1e-10, precision=glls.PREC_MIXED, use_graph=use_graph))
        assert st.status == glls.OK and np.isfinite(u).all()
    prob.close()
