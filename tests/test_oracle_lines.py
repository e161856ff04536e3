"""Pins for line systems and cyclic reduction (Def. 3.1/3.2, Algorithm 1,
Prop. 3.7, Thm. 3.8, Cor. 3.9)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import gll, lines
from oracle.discretize import Level
from oracle.fem import line_band_from_matrix, q1_stiffness
from paper_2504_10710_gb300 import inputs


def level_of(wl):
    xi, _ = gll.gll(wl.order)
    return Level(wl.dim, wl.nelem, wl.order, wl.coords(xi))


def random_tridiag(rng, shape, dominant=True):
    n = shape[-1]
    l = rng.standard_normal(shape)
    u = rng.standard_normal(shape)
    a = rng.standard_normal(shape) + (np.abs(l) + np.abs(u) + 0.5 if dominant else 0.0)
    l[..., 0] = 0.0
    u[..., -1] = 0.0
    return a, l, u


@pytest.mark.parametrize("n", list(range(1, 20)) + [31, 32, 33, 63, 64, 100, 127, 511])
def test_cr_equals_dense_lu_thomas_and_literal_algorithm1(n):
    rng = np.random.default_rng(n)
    a, l, u = random_tridiag(rng, (n,))
    g = rng.standard_normal(n)
    T = np.diag(a) + np.diag(l[1:], -1) + np.diag(u[:-1], 1)
    x_ref = sla.solve(T, g)
    x = lines.cr_solve(a, l, u, g)
    np.testing.assert_allclose(x, x_ref, atol=1e-12 * np.abs(x_ref).max())
    np.testing.assert_allclose(lines.thomas(a, l, u, g), x_ref, atol=1e-12 * np.abs(x_ref).max())
    if n <= 64:
        np.testing.assert_allclose(lines.cr_algorithm1(a, l, u, g), x_ref, atol=1e-12 * np.abs(x_ref).max())


def test_cr_vectorised_over_lines_matches_banded_solver():
    rng = np.random.default_rng(7)
    a, l, u = random_tridiag(rng, (6, 5, 37))
    g = rng.standard_normal((6, 5, 37))
    x = lines.cr_solve(a, l, u, g)
    for i in range(6):
        for j in range(5):
            ab = np.zeros((3, 37))
            ab[0, 1:] = u[i, j, :-1]
            ab[1] = a[i, j]
            ab[2, :-1] = l[i, j, 1:]
            np.testing.assert_allclose(x[i, j], sla.solve_banded((1, 1), ab, g[i, j]), atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 6, 9, 16, 25])
def test_two_level_step_is_exact_and_schur_complement_matches_prop37(n):
    """Thm. 3.8: one Richardson step preconditioned by Algorithm 1 with an
    exact coarse solve M0^-1 = (D - C A^-1 B)^-1 has zero error.  The coarse
    tridiagonal entries (Prop. 3.7, explicit product form) equal the Schur
    complement computed with a dense solve."""
    rng = np.random.default_rng(100 + n)
    a, l, u = random_tridiag(rng, (n,))
    T, Sinv, P, R, M0 = lines.algorithm1_operators(a, l, u)
    f = rng.standard_normal(n)
    x = Sinv @ f
    y = x + P @ np.linalg.solve(M0, R @ (f - T @ x))
    np.testing.assert_allclose(y, np.linalg.solve(T, f), atol=1e-12)
    # Prop. 3.7 entries for even i (1-based): a', l', u'
    ev = np.arange(1, n, 2)
    for k, i in enumerate(ev):
        ap = a[i] - l[i] * u[i - 1] / a[i - 1] - (u[i] * l[i + 1] / a[i + 1] if i + 1 < n else 0.0)
        assert abs(M0[k, k] - ap) < 1e-12
        if k > 0:
            assert abs(M0[k, k - 1] - (-l[i] * l[i - 1] / a[i - 1])) < 1e-12
        if k + 1 < len(ev):
            assert abs(M0[k, k + 1] - (-u[i] * u[i + 1] / a[i + 1])) < 1e-12
    # R = P^T and the Lemma 3.4 identity M^-1 = S^-1 + P M0^-1 R (I - M S^-1)
    Minv = Sinv + P @ np.linalg.solve(M0, R @ (np.eye(n) - T @ Sinv))
    np.testing.assert_allclose(Minv, np.linalg.inv(T), atol=1e-11)


def test_cr_block_toeplitz_matches_bgn_reduced_system():
    """Lemma A.2 (Buzbee-Golub-Nielson): for the scalar Toeplitz case A, T
    commuting, the even unknowns satisfy (2T^2 - A^2) x_2k + T^2 (x_2k-2 +
    x_2k+2) = T (y_2k-1 + y_2k+1) - A y_2k (the right-hand side read with y
    for the printed x)."""
    n = 15
    A, Tt = 4.0, -1.0
    a = np.full(n, A)
    l = np.full(n, Tt)
    u = np.full(n, Tt)
    l[0] = u[-1] = 0.0
    y = np.random.default_rng(3).standard_normal(n)
    x = lines.cr_solve(a, l, u, y)
    for i in range(1, n, 2):            # 1-based even indices i+1
        lhs = (2 * Tt ** 2 - A ** 2) * x[i] + Tt ** 2 * ((x[i - 2] if i >= 2 else 0) + (x[i + 2] if i + 2 < n else 0))
        rhs = Tt * (y[i - 1] + y[i + 1]) - A * y[i]
        assert abs(lhs - rhs) < 1e-12


CASES = [inputs.random2d((3, 2), 4, amp=0.1, seed=1), inputs.random2d((2, 3), 3, amp=0.15, seed=2),
         inputs.random3d((2, 2, 1), 3, amp=0.15, seed=3)]
BLOCK_CASES = CASES + [inputs.random2d((1, 1), 6, amp=0.1, seed=6), inputs.random3d((2, 1, 3), 4, amp=0.1, seed=7)]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_line_band_equals_assembled_entries(wl):
    lv = level_of(wl)
    A = lv.assemble()
    for s in range(lv.dim):
        a, l, u = lines.line_band(lv, s)
        a2, l2, u2 = line_band_from_matrix(lv, A, s)
        np.testing.assert_allclose(a, a2, atol=1e-12 * np.abs(a2).max())
        np.testing.assert_allclose(l, l2, atol=1e-12 * np.abs(a2).max())
        np.testing.assert_allclose(u, u2, atol=1e-12 * np.abs(a2).max())


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_line_preconditioner_inverts_band_on_each_line(wl):
    """B_s^-1 (B_s y) = y where B_s is the block-diagonal matrix of line
    systems (band 1 of A along every interior line, Def. 3.2)."""
    lv = level_of(wl)
    A = lv.assemble().tolil()
    ii = set(lv.interior_index().tolist())
    strides = np.cumprod((1,) + lv.shape[::-1])[:-1][::-1]
    for s in range(lv.dim):
        st = int(strides[lv.dim - 1 - s])
        B = np.zeros((lv.N, lv.N))
        for n in ii:
            B[n, n] = A[n, n]
            for m in (n - st, n + st):
                if m in ii:
                    B[n, m] = A[n, m]
        y = np.where(lv.interior, np.random.default_rng(s).standard_normal(lv.shape), 0.0)
        sm = lines.LineSmoother(lv, s)
        np.testing.assert_allclose(sm.apply_inverse((B @ y.ravel()).reshape(lv.shape)), y, atol=1e-11)


def test_fem_matrix_undeformed_is_q1_stencil():
    """On an undeformed uniform grid (p = 1, so GLL nodes are uniform) the
    bilinear FEM matrix is the classical 9-point Q1 stencil 8/3, -1/3."""
    wl = inputs.Workload("sq", 2, (4, 4), 1, inputs.identity_map, [], inputs._zero)
    lv = level_of(wl)
    A = q1_stiffness(lv).toarray()
    c = 2 * 5 + 2
    row = A[c].reshape(5, 5)
    np.testing.assert_allclose(row[1:4, 1:4], [[-1 / 3] * 3, [-1 / 3, 8 / 3, -1 / 3], [-1 / 3] * 3], atol=1e-14)


# ---- Def. 3.2 read literally: the line blocks R_L A P_L ---------------------
def _dense_line_blocks(lv, A, s):
    Ad = A.toarray()
    return [Ad[np.ix_(rows, rows)] for rows in lines.line_nodes(lv, s)]


def _from_band(ab, w):
    n = ab.shape[-1]
    T = np.zeros((n, n))
    for o in range(w + 1):
        T[np.arange(n - o), np.arange(o, n)] = ab[w - o, o:]
        T[np.arange(o, n), np.arange(n - o)] = ab[w - o, o:]
    return T


@pytest.mark.parametrize("wl", BLOCK_CASES, ids=lambda w: w.name)
def test_line_block_band_holds_the_whole_block(wl):
    """No entry of R_L A P_L lies farther than p from its diagonal: the banded
    copies, read from the assembled A and summed from the element matrices,
    both equal the principal submatrix of the assembled A on every line."""
    lv = level_of(wl)
    A = lv.assemble()
    for s in range(lv.dim):
        ab, w = lines.line_block_bands(lv, s, A)
        ab2, w2 = lines.line_block_bands(lv, s)
        assert w2 == w
        for k, T in enumerate(_dense_line_blocks(lv, A, s)):
            np.testing.assert_allclose(_from_band(ab[k], w), T, atol=1e-13 * np.abs(T).max())
            np.testing.assert_allclose(_from_band(ab2[k], w), T, atol=1e-13 * np.abs(T).max())


def _assembled_1d(ne, p):
    """Assembled 1-D reference stiffness K = D^T W D and weights W on ne
    elements (global 1-D grid of ne p + 1 nodes)."""
    xi, rho = gll.gll(p)
    D = gll.derivative_matrix(xi)
    Ke = D.T @ np.diag(rho) @ D
    n = ne * p + 1
    K = np.zeros((n, n))
    W = np.zeros(n)
    for e in range(ne):
        sl = slice(e * p, e * p + p + 1)
        K[sl, sl] += Ke
        W[sl] += rho
    return K, W


@pytest.mark.parametrize("dim,nelem,p", [(2, (3, 2), 4), (2, (1, 1), 7), (3, (2, 1, 2), 3)])
def test_line_block_of_a_box_grid_is_the_kronecker_closed_form(dim, nelem, p):
    """Undeformed box elements of sides h_a: A is the sum over axes a of
    c_a (K_a along a) x (W along the other axes) with c_a = prod_{b != a} h_b
    / h_a * 2^(2 - d) (the Jacobian and metric of the affine map), so the
    line block along axis s at fixed other indices m_b is
    c_s prod_b W_b[m_b] K_s[int, int] + sum_{a != s} c_a K_a[m_a, m_a]
    prod_{b != a, s} W_b[m_b] W_s[int].  Side lengths differ per axis, so a
    transposed axis fails."""
    scale = (2.0, 0.5, 1.5)[:dim]
    mp = lambda *X: tuple(scale[a] * X[a] for a in range(dim))
    wl = inputs.Workload("box", dim, nelem, p, mp, [], inputs._zero)
    lv = level_of(wl)
    A = lv.assemble()
    h = [scale[a] / nelem[a] for a in range(dim)]
    c = [np.prod([h[b] for b in range(dim) if b != a]) / h[a] * 2.0 ** (2 - dim) for a in range(dim)]
    KW = [_assembled_1d(nelem[a], p) for a in range(dim)]
    for s in range(dim):
        blocks = _dense_line_blocks(lv, A, s)
        others = [a for a in range(dim) if a != s]
        # interior indices of the other axes, slowest axis first (line order)
        grids = np.meshgrid(*[np.arange(1, nelem[a] * p) for a in reversed(others)], indexing="ij")
        idx = [g.ravel() for g in grids]
        m = {a: idx[len(others) - 1 - j] for j, a in enumerate(others)}
        Ks, Ws = KW[s]
        inner = slice(1, -1)
        for k, T in enumerate(blocks):
            ref = c[s] * np.prod([KW[b][1][m[b][k]] for b in others]) * Ks[inner, inner]
            for a in others:
                wprod = np.prod([KW[b][1][m[b][k]] for b in others if b != a])
                ref = ref + c[a] * KW[a][0][m[a][k], m[a][k]] * wprod * np.diag(Ws[inner])
            np.testing.assert_allclose(T, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_fem_line_blocks_are_tridiagonal(wl):
    """R_L A~ P_L of the bilinear FEM matrix has no coupling beyond the
    neighbours along the line: the two readings of Def. 3.2 coincide there."""
    lv = level_of(wl)
    At = q1_stiffness(lv)
    for s in range(lv.dim):
        a, l, u = (z.reshape(-1, z.shape[-1]) for z in line_band_from_matrix(lv, At, s))
        for k, T in enumerate(_dense_line_blocks(lv, At, s)):
            tri = np.diag(a[k]) + np.diag(l[k][1:], -1) + np.diag(u[k][:-1], 1)
            np.testing.assert_allclose(T, tri, atol=1e-13 * np.abs(T).max())


@pytest.mark.parametrize("wl", CASES + [inputs.random2d((4, 3), 1, amp=0.1, seed=5)], ids=lambda w: w.name)
def test_block_line_preconditioner_inverts_each_line_block(wl):
    """B_s^-1 (B_s y) = y with B_s the block-diagonal matrix of the line
    blocks R_L A P_L (every coupling between two nodes of the same interior
    line along s); at p = 1 it is the band-1 preconditioner."""
    lv = level_of(wl)
    A = lv.assemble()
    Ad = A.toarray()
    for s in range(lv.dim):
        B = np.zeros_like(Ad)
        for rows in lines.line_nodes(lv, s):
            B[np.ix_(rows, rows)] = Ad[np.ix_(rows, rows)]
        y = np.where(lv.interior, np.random.default_rng(s).standard_normal(lv.shape), 0.0)
        sm = lines.BlockLineSmoother(lv, s, A)
        np.testing.assert_allclose(sm.apply_inverse((B @ y.ravel()).reshape(lv.shape)), y, atol=1e-11)
        if lv.p == 1:
            g = np.where(lv.interior, np.random.default_rng(7 + s).standard_normal(lv.shape), 0.0)
            np.testing.assert_allclose(sm.apply_inverse(g), lines.LineSmoother(lv, s).apply_inverse(g), atol=1e-12)
