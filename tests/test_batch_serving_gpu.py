"""Batched solves of uneven problems in one graph launch, and the serving loop
(admission by HBM budget, concurrent requests): results equal those of single
solves, alone or in the mix."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_10710_gb300 import glls, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


# uneven grids, orders and dimensions; all converge in 12-17 FCG iterations
MIX = [inputs.random2d((9, 7), 6, amp=0.1, seed=21), inputs.random2d((16, 16), 8, amp=0.1, seed=22),
       inputs.random2d((4, 5), 7, amp=0.05, seed=23), inputs.random3d((3, 3, 2), 4, amp=0.1, seed=24),
       inputs.random2d((10, 6), 4, amp=0.1, seed=25), inputs.random2d((6, 8), 5, amp=0.1, seed=26)]


def _setup(wl):
    prob, coords = glls.problem_for(wl)
    f = wl.sample_rhs(coords)[0]
    g = wl.sample_dirichlet(coords)
    prob.set_rhs(f)
    prob.set_dirichlet(g)
    return prob, coords, f, g


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
def test_solve_batch_equals_single_solves(prec):
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=prec, max_iter=300)
    probs = [_setup(wl)[0] for wl in MIX]
    single, its = [], []
    for p in probs:
        u = np.zeros(p.N)
        its.append(p.solve(u, o).iterations)
        single.append(u)
    for _ in range(2):          # second launch reuses the cached batch graph
        outs = [np.zeros(p.N) for p in probs]
        stats = glls.solve_batch(probs, outs, o)
        for u, ub, st, k in zip(single, outs, stats, its):
            assert _rel(ub, u) < 1e-10
            assert abs(st.iterations - k) <= 1
            assert st.status == glls.OK and st.rel_residual <= 1e-10
    for p in probs:
        p.close()


def test_estimate_bytes_tracks_allocation():
    for wl in MIX:
        prob, coords, _, _ = _setup(wl)
        est = glls.estimate_bytes(wl.dim, wl.nelem, wl.order, coords)
        actual = prob.info.device_bytes
        assert 0.8 * actual <= est <= 1.25 * actual, (wl.name, est, actual)
        prob.close()


def _request(wl):
    xi, _ = glls.gll(wl.order)
    coords = wl.coords(xi)
    return coords, wl.sample_rhs(coords)[0], wl.sample_dirichlet(coords)


def test_server_results_same_alone_and_in_the_mix():
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5, precision=glls.PREC_MIXED)
    srv = glls.Server(budget_bytes=8 << 30, slots=4)
    reqs = [(wl,) + _request(wl) for wl in MIX]
    alone = []
    for wl, coords, f, g in reqs:                    # one at a time
        out = np.zeros(f.size)
        t = srv.submit(wl.dim, wl.nelem, wl.order, coords, f, g, o, out)
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK
        alone.append(out)
    outs, tickets = [], []
    for rep in range(3):                             # all at once, three times
        for wl, coords, f, g in reqs:
            out = np.zeros(f.size)
            outs.append(out)
            tickets.append(srv.submit(wl.dim, wl.nelem, wl.order, coords, f, g, o, out))
    for t in tickets:
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK and stats.rel_residual <= 1e-10
    for k, out in enumerate(outs):
        assert _rel(out, alone[k % len(reqs)]) < 1e-10
    inf = srv.info()
    assert inf.completed == len(reqs) * 4 and inf.failed == 0
    assert inf.cached_problems >= len(reqs)        # meshes stay resident
    srv.close()


def test_server_admission_by_budget_and_eviction():
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5)
    a, b = MIX[1], MIX[2]
    ra, rb = _request(a), _request(b)
    ea = glls.estimate_bytes(a.dim, a.nelem, a.order, ra[0])
    eb = glls.estimate_bytes(b.dim, b.nelem, b.order, rb[0])
    # room for either mesh but not both: alternating requests force eviction
    srv = glls.Server(budget_bytes=int(1.05 * max(ea, eb)) + (ea + eb) // 10, slots=2)
    tickets, outs = [], []
    for k in range(6):
        wl, (coords, f, g) = (a, ra) if k % 2 == 0 else (b, rb)
        out = np.zeros(f.size)
        outs.append((k % 2, out))
        tickets.append(srv.submit(wl.dim, wl.nelem, wl.order, coords, f, g, o, out))
    for t in tickets:
        st, _ = srv.poll(t, wait=True)
        assert st == glls.OK
    assert srv.info().resident_bytes <= srv.info().budget_bytes
    ref = {0: outs[0][1], 1: outs[1][1]}
    for which, out in outs:
        assert _rel(out, ref[which]) < 1e-10
    # a request larger than the whole budget fails with GLLS_ERR_BUDGET
    small = glls.Server(budget_bytes=max(eb // 4, 1), slots=1)
    coords, f, g = rb
    out = np.zeros(f.size)
    t = small.submit(b.dim, b.nelem, b.order, coords, f, g, o, out)
    st, _ = small.poll(t, wait=True)
    assert st == glls.ERR_BUDGET
    small.close()
    srv.close()


def test_server_poll_without_waiting():
    o = glls.opts()
    wl = MIX[1]
    coords, f, g = _request(wl)
    srv = glls.Server(budget_bytes=4 << 30, slots=1)
    out = np.zeros(f.size)
    t = srv.submit(wl.dim, wl.nelem, wl.order, coords, f, g, o, out)
    st, stats = srv.poll(t, wait=False)
    deadline = time.time() + 60
    while st == glls.NOT_READY and time.time() < deadline:
        time.sleep(0.005)
        st, stats = srv.poll(t, wait=False)
    assert st == glls.OK and stats.iterations > 0
    srv.close()


@pytest.mark.parametrize("smoother", [glls.SMOOTHER_GLL, glls.SMOOTHER_GLL_BAND1], ids=["blocks", "band1"])
def test_autotune_picks_valid_tiles_and_keeps_results(smoother):
    wl = MIX[1]
    prob, coords = glls.problem_for(wl, smoother)
    f, g = wl.sample_rhs(coords)[0], wl.sample_dirichlet(coords)
    prob.set_rhs(f)
    prob.set_dirichlet(g)
    o = glls.opts(tol=1e-10, gamma=1, alpha=0.5)
    before = np.zeros(prob.N)
    st0 = prob.solve(before, o)
    tiles = prob.autotune()
    # GLL line blocks: 0 (launch heuristic) or 1..16 lines per CTA
    assert tiles and all(c in (0, 1, 2, 4, 8, 16) and us > 0 for c, us in tiles.values())
    after = np.zeros(prob.N)
    st1 = prob.solve(after, o)            # graphs are re-captured with the chosen tiles
    assert _rel(after, before) < 1e-10 and abs(st1.iterations - st0.iterations) <= 1
    assert st1.kernels > st1.iterations * 10
    prob.close()


@pytest.mark.parametrize("smoother,alpha", [(glls.SMOOTHER_GLL, 2.0 / 3.0), (glls.SMOOTHER_FEM, 0.16)],
                         ids=["gll_blocks", "fem"])
def test_uneven_batch_sample(smoother, alpha):
    """A sample of the batched uneven workload (n x n elements, n in 4..64,
    p in 4..12, amplitude up to 0.2), including its hardest draws (p = 12 and
    amplitude near 0.2): with the GLL line blocks (alpha = 2/3) and with the
    FEM line smoother (alpha = 0.16) every problem reaches 1e-10 in the
    batch, with the single solves' results."""
    ws = inputs.batch_uneven()
    pick = [w for w in ws if w.order == 12 and w.params["amp"] > 0.17][:2] + ws[:4]
    o = glls.opts(tol=1e-10, gamma=1, alpha=alpha, precision=glls.PREC_MIXED, max_iter=300)
    probs, single = [], []
    for w in pick:
        prob, coords = glls.problem_for(w, smoother)
        prob.set_rhs(w.sample_rhs(coords)[0])
        prob.set_dirichlet(w.sample_dirichlet(coords))
        u = np.zeros(prob.N)
        st = prob.solve(u, o)
        assert st.status == glls.OK and st.rel_residual <= 1e-10, w.name
        probs.append(prob)
        single.append((u, st.iterations))
    outs = [np.zeros(p.N) for p in probs]
    stats = glls.solve_batch(probs, outs, o)
    for (u, k), ub, st in zip(single, outs, stats):
        assert st.status == glls.OK and abs(st.iterations - k) <= 1
        assert _rel(ub, u) < 1e-9
    for p in probs:
        p.close()


def _alone(wl, coords, f, g, o):
    prob, _ = glls.problem_for(wl)
    prob.set_rhs(f)
    prob.set_dirichlet(g)
    u = np.zeros(prob.N)
    assert prob.solve(u, o).status == glls.OK
    prob.close()
    return u


def test_server_same_mesh_concurrent_requests_run_on_clones():
    """Requests for one mesh that arrive together run at once on clones of
    the resident problem (shared mesh data), each with its own right-hand
    side; every result equals the solve of that right-hand side alone."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    wl = inputs.random2d((32, 32), 8, amp=0.1, seed=27)
    coords, f, g = _request(wl)
    fs = [f * (1.0 + 0.5 * k) + k for k in range(4)]
    srv = glls.Server(budget_bytes=8 << 30, slots=4)
    outs = [np.zeros(f.size) for _ in fs]
    tickets = [srv.submit(wl.dim, wl.nelem, wl.order, coords, fk, g, o, out) for fk, out in zip(fs, outs)]
    for t in tickets:
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK and stats.rel_residual <= 1e-10
    inf = srv.info()
    assert inf.cached_problems == 1 and inf.clones >= 1 and inf.cached_instances == 1 + inf.clones
    srv.close()
    for fk, out in zip(fs, outs):
        assert _rel(out, _alone(wl, coords, fk, g, o)) < 1e-10


def test_server_eviction_while_other_meshes_are_busy():
    """Several slots and a budget that holds about two of four meshes: idle
    meshes are evicted while others are busy, and every result still equals
    its mesh's solve alone (admission hands a worker its problem, never an
    index that eviction can shift)."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    wls = [MIX[0], MIX[1], MIX[4], MIX[5]]
    reqs = [(wl,) + _request(wl) for wl in wls]
    est = [glls.estimate_bytes(wl.dim, wl.nelem, wl.order, c) for wl, c, _, _ in reqs]
    alone = [_alone(wl, c, f, g, o) for wl, c, f, g in reqs]
    srv = glls.Server(budget_bytes=int(2.2 * max(est)), slots=3)
    order = np.random.default_rng(5).integers(0, len(reqs), 24)
    outs, tickets = [], []
    for k in order:
        wl, c, f, g = reqs[k]
        out = np.zeros(f.size)
        outs.append((k, out))
        tickets.append(srv.submit(wl.dim, wl.nelem, wl.order, c, f, g, o, out))
    for t in tickets:
        st, _ = srv.poll(t, wait=True)
        assert st == glls.OK
    inf = srv.info()
    assert inf.completed == len(order) and inf.resident_bytes <= inf.budget_bytes
    srv.close()
    for k, out in outs:
        assert _rel(out, alone[k]) < 1e-10


def test_server_cancel_queued_request():
    """A queued request can be cancelled (its output is never written); a
    running one cannot; unknown tickets are rejected."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_FP64)
    wl = inputs.random2d((48, 48), 8, amp=0.1, seed=28)
    coords, f, g = _request(wl)
    srv = glls.Server(budget_bytes=8 << 30, slots=1)
    outs = [np.zeros(f.size) for _ in range(3)]
    tickets = [srv.submit(wl.dim, wl.nelem, wl.order, coords, f, g, o, out) for out in outs]
    deadline = time.time() + 60
    while srv.info().running == 0 and time.time() < deadline:
        time.sleep(0.001)
    assert srv.cancel(tickets[2]) == glls.OK
    assert srv.cancel(tickets[2]) == glls.ERR_INVALID
    assert srv.cancel(12345678) == glls.ERR_INVALID
    assert srv.cancel(tickets[0]) == glls.NOT_READY      # running (or finished, not yet polled)
    for t in tickets[:2]:
        st, _ = srv.poll(t, wait=True)
        assert st == glls.OK
    assert not outs[2].any()
    assert srv.info().completed == 2
    srv.close()


def test_server_registered_meshes_match_single_solves():
    """Meshes registered once and solved by id (the request reads the caller's
    f and g when it runs): results equal single solves; the first request on
    a mesh reports its set-up (setup_kind 1), concurrent ones on the same
    mesh a clone (2) or a resident instance (0); queue time is within the
    latency."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    wls = [MIX[0], MIX[3], MIX[2]]
    reqs = [(wl,) + _request(wl) for wl in wls]
    srv = glls.Server(budget_bytes=8 << 30, slots=3)
    ids = [srv.register(wl.dim, wl.nelem, wl.order, c) for wl, c, _, _ in reqs]
    assert len(set(ids)) == len(ids)
    fs = {k: [f * (1.0 + 0.25 * j) for j in range(3)] for k, (_, _, f, _) in enumerate(reqs)}
    outs, tickets = [], []
    for j in range(3):
        for k, (wl, c, f, g) in enumerate(reqs):
            out = np.full(f.size, np.nan)
            outs.append((k, j, out))
            tickets.append(srv.submit_mesh(ids[k], fs[k][j], g, o, out))
    kinds = {k: [] for k in range(len(reqs))}
    for (k, j, _), t in zip(outs, tickets):
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK and stats.rel_residual <= 1e-10
        assert 0.0 <= stats.queue_ms <= stats.solve_ms
        kinds[k].append(stats.setup_kind)
        if stats.setup_kind:
            assert stats.setup_ms > 0.0
    for k in kinds:
        assert kinds[k].count(1) == 1 and set(kinds[k]) <= {0, 1, 2}
    with pytest.raises(glls.GllsError):
        srv.submit_mesh(987654, reqs[0][2], None, o, np.zeros(reqs[0][2].size))
    srv.close()
    for k, j, out in outs:
        wl, c, _, g = reqs[k]
        assert _rel(out, _alone(wl, c, fs[k][j], g, o)) < 1e-10


@pytest.mark.parametrize("prec", [glls.PREC_MIXED, glls.PREC_FP64], ids=["mixed", "fp64"])
def test_server_groups_same_mesh_requests_into_one_multi_rhs_solve(prec):
    """With grouping on, queued requests of one resident mesh with the same
    Dirichlet data are solved together as one multi-right-hand-side solve
    (group sizes are powers of two); each result equals its solve alone."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec)
    wl = MIX[1]
    coords, f, g = _request(wl)
    srv = glls.Server(budget_bytes=8 << 30, slots=1)
    srv.set_max_group(4)
    mid = srv.register(wl.dim, wl.nelem, wl.order, coords)
    fs = [f * (1.0 + 0.3 * j) - 0.1 * j for j in range(7)]
    outs = [np.full(f.size, np.nan) for _ in fs]
    tickets = [srv.submit_mesh(mid, fk, g, o, out) for fk, out in zip(fs, outs)]
    groups = []
    for t in tickets:
        st, stats = srv.poll(t, wait=True)
        assert st == glls.OK and stats.rel_residual <= 1e-10
        groups.append(stats.group)
    inf = srv.info()
    srv.close()
    assert set(groups) <= {1, 2, 4} and max(groups) > 1, groups
    assert inf.grouped == sum(1 for k in groups if k > 1)
    for fk, out in zip(fs, outs):
        assert _rel(out, _alone(wl, coords, fk, g, o)) < 1e-10


# uneven 2-D problems: several order chains (8-4-2-1, 6-3-1, 5-2-1, 4-2-1),
# two of them with more than one problem, ragged element counts,
# and orders above 8 (the run-time-order line-block instance: 12-6-3-1 and
# 10-5-2-1 next to 5-2-1)
WORKLIST = [inputs.random2d((9, 7), 6, amp=0.1, seed=61), inputs.random2d((16, 12), 8, amp=0.15, seed=62),
            inputs.random2d((4, 5), 5, amp=0.05, seed=63), inputs.random2d((10, 6), 4, amp=0.1, seed=64),
            inputs.random2d((6, 8), 6, amp=0.1, seed=65), inputs.random2d((21, 19), 8, amp=0.1, seed=66),
            inputs.random2d((3, 2), 5, amp=0.1, seed=67), inputs.random2d((7, 5), 12, amp=0.1, seed=68),
            inputs.random2d((5, 9), 10, amp=0.15, seed=69), inputs.random2d((4, 4), 12, amp=0.05, seed=70)]


@pytest.mark.parametrize("prec", [glls.PREC_FP64, glls.PREC_MIXED], ids=["fp64", "mixed"])
def test_worklist_batch_equals_single_solves(prec):
    """The work-list batch (one launch per step over all problems of an order
    chain) gives each problem its single-solve result and iteration count;
    a second call reuses the cached plan."""
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=prec)
    setups = [_setup(wl) for wl in WORKLIST]
    probs = [s[0] for s in setups]
    alone = []
    for prob in probs:
        u = np.zeros(prob.N)
        st = prob.solve(u, o)
        alone.append((u, st.iterations))
    for rep in range(2):
        outs = [np.full(p.N, np.nan) for p in probs]
        stats = glls.solve_batch(probs, outs, o, worklist=True)
        # FP64: the same kernels in the same order (up to the order of the
        # seam atomics); mixed: FP32 rounding of the cycle, as between two
        # single mixed solves
        tol = 1e-12 if prec == glls.PREC_FP64 else 1e-8
        for (u, its), out, st in zip(alone, outs, stats):
            assert st.status == glls.OK and st.rel_residual <= 1e-10
            assert abs(st.iterations - its) <= 1
            assert _rel(out, u) < tol
        assert stats[0].kernels > 0
    for p in probs:
        p.close()


def test_worklist_batch_device_outputs_and_refusals():
    o = glls.opts(tol=1e-10, gamma=1, alpha=2.0 / 3.0, precision=glls.PREC_MIXED)
    probs = [_setup(wl)[0] for wl in WORKLIST[:3]]
    outs = [torch.zeros(p.N, dtype=torch.float64, device="cuda") for p in probs]
    stats = glls.solve_batch(probs, outs, o, worklist=True)
    for p, out, st in zip(probs, outs, stats):
        u = np.zeros(p.N)
        p.solve(u, o)
        assert st.status == glls.OK and _rel(out.cpu().numpy(), u) < 1e-8
    # 3-D problems and GMRES are refused (the graph-branch batch takes them)
    p3 = _setup(inputs.random3d((3, 3, 2), 4, amp=0.1, seed=24))[0]
    with pytest.raises(glls.GllsError) as ei:
        glls.solve_batch([probs[0], p3], [np.zeros(probs[0].N), np.zeros(p3.N)], o, worklist=True)
    assert ei.value.status == glls.ERR_INVALID
    with pytest.raises(glls.GllsError):
        glls.solve_batch(probs, [np.zeros(p.N) for p in probs],
                         glls.opts(tol=1e-10, krylov=glls.KRYLOV_GMRES), worklist=True)
    for p in probs + [p3]:
        p.close()
