"""Line systems (Def. 3.1, Def. 3.2), cyclic reduction as a direct multigrid
(Algorithm 1, Prop. 3.7, Thm. 3.8, Cor. 3.9) and the damped line-smoothing
step of Algorithm 2.  Test infrastructure only.

Def. 3.2 writes the line system of a grid line L as R_L A_p P_L, the
principal submatrix of the assembled stiffness on L's interior nodes, while
its surrounding text calls the systems tridiagonal.  Both readings are here:

  * ``BlockLineSmoother`` (the default GLL smoother): R_L A_p P_L taken
    literally.  Two nodes of a line couple only through an element that holds
    both, and an element spans p intervals of the line, so the block has
    half-bandwidth p; it is kept in banded storage and solved by a banded
    Cholesky factorisation (a library routine).  With this reading the GLL
    column of Table 1 (problem 1) is reproduced at p_L = 8 .. 64.
  * ``LineSmoother`` on ``line_band`` (option ``gll_band1``): the band-1 part
    [A]^(1) restricted to the line (Def. 3.1 with half-bandwidth 1), i.e.
    the diagonal and the couplings to the two neighbours along the line,
    solved by cyclic reduction.

For the FEM matrix A~_p (bilinear elements on the GLL nodes) a node couples
only to its neighbours along a line, so R_L A~_p P_L is tridiagonal and both
readings coincide.  On a multi-element grid the lines are the global grid
lines, running through all elements.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .discretize import Level, apply_1d


# --------------------------------------------------------------------------
# band-1 entries of the assembled stiffness matrix
# --------------------------------------------------------------------------
def _axis_vec(level: Level, v, a, length=None):
    """Broadcast a 1-D vector along element-local axis a."""
    d = level.dim
    shape = [1] * (2 * d)
    shape[level.eaxis(a)] = len(v) if length is None else length
    return np.asarray(v).reshape(shape)


def _slice_axis(arr, axis, sl):
    idx = [slice(None)] * arr.ndim
    idx[axis] = sl
    return arr[tuple(idx)]


def band_diagonal(level: Level):
    """A[n, n] for every node n, assembled.

    Element part, from eq. (discreteBilinear) with the nodal basis:
      sum_a sum_q G_aa(q) D[q, m_a]^2   (q runs along axis a through m)
      + sum_{a != b} G_ab(m) D[m_a, m_a] D[m_b, m_b]."""
    d, D = level.dim, level.D
    Dd = np.diag(D)
    De = np.zeros(level.eshape)
    for a in range(d):
        De += apply_1d((D * D).T, level.G[a, a], level.eaxis(a))
        for b in range(d):
            if b != a:
                De += level.G[a, b] * _axis_vec(level, Dd, a) * _axis_vec(level, Dd, b)
    return level.from_elements(De)


def band_offdiag(level: Level, s: int):
    """A[n, n + e_s] for every node n with a neighbour n + e_s along axis s,
    assembled; returned on the grid with axis s shortened by one (entry at n).

    Element part for local m (m_s < p):
      sum_q G_ss(q) D[q, m_s] D[q, m_s+1]                       (a = b = s)
      + sum_{b != s} G_sb(m + e_s) D[m_s+1, m_s] D[m_b, m_b]     (a = s, b != s)
      + sum_{a != s} G_as(m) D[m_a, m_a] D[m_s, m_s+1]           (a != s, b = s)
    (terms with a = b != s vanish: they need q_s = m_s and q_s = m_s + 1)."""
    d, D, p = level.dim, level.D, level.p
    Dd = np.diag(D)
    ax = level.eaxis(s)
    M1 = (D[:, :-1] * D[:, 1:]).T           # M1[m, q] = D[q, m] D[q, m+1], m < p
    Oe = apply_1d(M1, level.G[s, s], ax)
    sub = _axis_vec(level, np.diag(D, -1), s, p)   # D[m_s+1, m_s]
    sup = _axis_vec(level, np.diag(D, 1), s, p)    # D[m_s, m_s+1]
    for b in range(d):
        if b == s:
            continue
        Db = _axis_vec(level, Dd, b)
        Oe = Oe + _slice_axis(level.G[s, b], ax, slice(1, None)) * sub * Db
        Oe = Oe + _slice_axis(level.G[b, s], ax, slice(0, p)) * sup * Db
    # scatter element couplings (m, m + e_s) onto the lower global node
    t = d - 1 - s
    shape = list(level.shape)
    shape[t] -= 1
    strides = np.cumprod((1,) + tuple(shape[::-1]))[:-1][::-1]
    lin = 0
    for tt in range(d):
        idx = level.gidx[tt]
        if tt == t:
            idx = _slice_axis(idx, d + t, slice(0, p))
        lin = lin + idx * int(strides[tt])
    lin = np.broadcast_to(lin, Oe.shape)
    out = np.bincount(lin.ravel(), weights=Oe.ravel(), minlength=int(np.prod(shape)))
    return out.reshape(shape)


def line_band(level: Level, s: int):
    """Tridiagonal systems of all interior grid lines along axis s.

    Returns (a, l, u) with shape (*other interior dims, n), n = N_s - 2, axis s
    moved last: a_k = A[k, k], l_k = A[k, k-1], u_k = A[k, k+1] along the line
    (l_0 = u_{n-1} = 0: boundary nodes are Dirichlet, not unknowns)."""
    d = level.dim
    t = d - 1 - s
    diag = band_diagonal(level)
    off = band_offdiag(level, s)
    inner = tuple(slice(1, -1) for _ in range(d))
    a = np.moveaxis(diag[inner], t, -1)
    # couplings between interior nodes k and k+1 (global k = 1..N_s-3)
    sl = [slice(1, -1)] * d
    sl[t] = slice(1, None)          # lower node 1 .. N_s-2 (off has N_s-1 entries)
    o = np.moveaxis(off[tuple(sl)], t, -1)   # o[..., j] couples interior j and j+1
    n = a.shape[-1]
    u = np.zeros_like(a)
    l = np.zeros_like(a)
    u[..., :n - 1] = o[..., :n - 1]
    l[..., 1:] = o[..., :n - 1]
    return a, l, u


# --------------------------------------------------------------------------
# cyclic reduction
# --------------------------------------------------------------------------
def cr_solve(a, l, u, g):
    """Solve the tridiagonal systems T x = g (vectorised over leading axes) by
    the direct multigrid of Cor. 3.9.  With 1-based indices, odd unknowns are
    the fine points and even ones the coarse points (Def. 3.6).  One level is
    Algorithm 1 with the operators of Thm. 3.8:
      x = S^-1 g                    (x_odd = g_odd / a_odd, x_even = 0)
      c = R (g - T x)               (residual vanishes at odd rows; R = P^T
                                     then just picks the even rows)
      e = T0^-1 c                   (T0 = D - C A^-1 B, Prop. 3.7, recursive)
      y = x + P e                   (even: e; odd: -= (l/a) e_left + (u/a) e_right)
    T0 entries for even i (Prop. 3.7 with the diagonal read from the explicit
    product C A^-1 B):
      a'_i = a_i - l_i u_{i-1}/a_{i-1} - u_i l_{i+1}/a_{i+1}
      l'_i = -l_i l_{i-1}/a_{i-1},  u'_i = -u_i u_{i+1}/a_{i+1}."""
    n = a.shape[-1]
    if n == 1:
        return g / a
    # 0-based k: 1-based odd i = k+1 are k = 0, 2, 4 ...; 1-based even are k = 1, 3, ...
    ao, lo, uo, go = a[..., 0::2], l[..., 0::2], u[..., 0::2], g[..., 0::2]
    ae, le, ue, ge = a[..., 1::2], l[..., 1::2], u[..., 1::2], g[..., 1::2]
    no, nc = ao.shape[-1], ae.shape[-1]

    def padded(z, fill):
        # odd-point arrays extended to nc + 1 entries so that coarse point j has
        # its left odd neighbour at j and its right one at j + 1; a missing
        # right neighbour (n even) only meets u = 0 of the last unknown.
        if z.shape[-1] == nc + 1:
            return z
        return np.concatenate([z, np.full_like(z[..., :1], fill)], axis=-1)

    xo = go / ao                                           # x = S^-1 g
    xo_p = padded(xo, 0.0)
    c = ge - le * xo_p[..., :nc] - ue * xo_p[..., 1:]      # c = R (g - T x)
    ap, lp, up = padded(ao, 1.0), padded(lo, 0.0), padded(uo, 0.0)
    a0 = ae - le * up[..., :nc] / ap[..., :nc] - ue * lp[..., 1:] / ap[..., 1:]
    l0 = -le * lp[..., :nc] / ap[..., :nc]
    u0 = -ue * up[..., 1:] / ap[..., 1:]
    e = cr_solve(a0, l0, u0, c)                            # e = T0^-1 c
    zero = np.zeros_like(e[..., :1])
    eleft = np.concatenate([zero, e], axis=-1)[..., :no]   # coarse point left of odd j
    eright = np.concatenate([e, zero], axis=-1)[..., :no]  # coarse point right of odd j
    x = np.empty_like(g)
    x[..., 1::2] = e                                       # y = x + P e
    x[..., 0::2] = xo - (lo / ao) * eleft - (uo / ao) * eright
    return x


def algorithm1_operators(a, l, u):
    """Explicit dense S^-1, P, R = P^T and coarse M0 of Thm. 3.8 for one scalar
    tridiagonal matrix (1-D arrays a, l, u; l[0] = u[-1] = 0)."""
    n = len(a)
    T = np.diag(a) + np.diag(l[1:], -1) + np.diag(u[:-1], 1)
    odd = np.arange(0, n, 2)     # 1-based odd
    even = np.arange(1, n, 2)    # 1-based even (coarse)
    Sinv = np.zeros((n, n))
    Sinv[odd, odd] = 1.0 / a[odd]
    P = np.zeros((n, len(even)))
    for k, i in enumerate(even):
        P[i, k] = 1.0
        P[i - 1, k] = -u[i - 1] / a[i - 1]          # -A_{i-1}^-1 U_{i-1}
        if i + 1 < n:
            P[i + 1, k] = -l[i + 1] / a[i + 1]      # -A_{i+1}^-1 L_{i+1}
    R = P.T
    # Schur complement D - C A^-1 B in the even unknowns (Prop. 3.7)
    Aoo = T[np.ix_(odd, odd)]
    B = T[np.ix_(odd, even)]
    C = T[np.ix_(even, odd)]
    Dm = T[np.ix_(even, even)]
    M0 = Dm - C @ np.linalg.solve(Aoo, B)
    return T, Sinv, P, R, M0


def cr_algorithm1(a, l, u, g):
    """Literal Algorithm 1 (two-level, no post-smoothing) applied recursively
    (Cor. 3.9), with the explicit matrices of Thm. 3.8; for small single lines."""
    n = len(a)
    if n == 1:
        return g / a
    T, Sinv, P, R, M0 = algorithm1_operators(a, l, u)
    x = Sinv @ g
    rc = R @ (g - T @ x)
    a0 = np.diag(M0).copy()
    l0 = np.concatenate([[0.0], np.diag(M0, -1)])
    u0 = np.concatenate([np.diag(M0, 1), [0.0]])
    return x + P @ cr_algorithm1(a0, l0, u0, rc)


def thomas(a, l, u, g):
    """Textbook Thomas algorithm (Gaussian elimination without pivoting),
    used only as an independent check of cyclic reduction."""
    n = len(a)
    c = np.zeros(n)
    d = np.zeros(n)
    c[0] = u[0] / a[0]
    d[0] = g[0] / a[0]
    for i in range(1, n):
        m = a[i] - l[i] * c[i - 1]
        c[i] = u[i] / m if i < n - 1 else 0.0
        d[i] = (g[i] - l[i] * d[i - 1]) / m
    x = np.zeros(n)
    x[-1] = d[-1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - c[i] * x[i + 1]
    return x


# --------------------------------------------------------------------------
# line preconditioner and smoothing step
# --------------------------------------------------------------------------
class LineSmoother:
    """B_s^-1 for the grid lines along axis s (Def. 3.2): block Jacobi over the
    lines, each block the tridiagonal line system solved by cyclic reduction."""

    def __init__(self, level: Level, s: int, band=None):
        self.level, self.s = level, s
        self.t = level.dim - 1 - s
        self.a, self.l, self.u = line_band(level, s) if band is None else band

    def apply_inverse(self, res):
        d = self.level.dim
        inner = tuple(slice(1, -1) for _ in range(d))
        g = np.moveaxis(np.asarray(res).reshape(self.level.shape)[inner], self.t, -1)
        x = cr_solve(self.a, self.l, self.u, g)
        out = np.zeros(self.level.shape)
        out[inner] = np.moveaxis(x, -1, self.t)
        return out

    def smooth(self, x, r, alpha):
        """x <- x + alpha B_s^-1 (r - A x)   (one step of Algorithm 2)."""
        return x + alpha * self.apply_inverse(r - self.level.apply(x))


# --------------------------------------------------------------------------
# Def. 3.2 read literally: the line block R_L A_p P_L
# --------------------------------------------------------------------------
def line_nodes(level: Level, s: int):
    """Global node indices of the interior nodes of every interior grid line
    along axis s: array (nlines, n), n = N_s - 2, the other axes' interior
    indices enumerated slowest first, nodes ordered along s."""
    d = level.dim
    t = d - 1 - s
    idx = np.arange(level.N).reshape(level.shape)
    inner = tuple(slice(1, -1) for _ in range(d))
    lin = np.moveaxis(idx[inner], t, -1)
    return lin.reshape(-1, lin.shape[-1])


def line_block_bands(level: Level, s: int, A=None, Ae=None):
    """R_L A P_L (Def. 3.2) of every interior grid line L along axis s.

    Returns (ab, w): LAPACK upper banded storage ab[line, w + i - j, j] =
    T_L[i, j] for j - w <= i <= j, with w = min(p, n - 1).  Entries of T_L
    farther than p from the diagonal are zero (no element spans more than p
    intervals of a line), so the band holds the whole block.

    With A (an assembled sparse stiffness) the entries are read from it.
    Otherwise they are assembled from the element matrices (``Ae``, or
    ``Level.element_matrices`` chunk by chunk): R_L A P_L = sum over the
    elements e of R_L Q_e^T A_e Q_e P_L, i.e. every entry of A_e between two
    local nodes that differ only in their s index, added at the two nodes'
    positions on their global line when both are interior unknowns of an
    interior line."""
    lin = line_nodes(level, s)
    nl, n = lin.shape
    w = min(level.p, n - 1)
    ab = np.zeros((nl, w + 1, n))
    if A is not None:
        A = A.tocsr()
        for o in range(w + 1):
            rows = lin[:, :n - o].ravel()
            cols = lin[:, o:].ravel()
            ab[:, w - o, o:] = np.asarray(A[rows, cols]).reshape(nl, n - o)
        return ab, w
    d, n1 = level.dim, level.p + 1
    n1d = n1 ** d
    line_of = np.full(level.N, -1)
    pos_of = np.full(level.N, -1)
    line_of[lin.ravel()] = np.repeat(np.arange(nl), n)
    pos_of[lin.ravel()] = np.tile(np.arange(n), nl)
    # local lines along s: element-local flat indices, (n1^(d-1), n1)
    loc = np.moveaxis(np.arange(n1d).reshape((n1,) * d), d - 1 - s, -1).reshape(-1, n1)
    glin = level.lin.reshape(-1, n1d)
    nE = glin.shape[0]
    chunk = max(1, int(2e7 // (n1d * n1d)))
    for e0 in range(0, nE, chunk):
        e1 = min(nE, e0 + chunk)
        Ablk = Ae[e0:e1] if Ae is not None else level.element_matrices(slice(e0, e1))
        gnode = glin[e0:e1][:, loc]                 # (ne, nloc_lines, n1) global nodes
        li = line_of[gnode]
        po = pos_of[gnode]
        for i in range(n1):
            for i2 in range(i, min(n1, i + w + 1)):
                vals = Ablk[:, loc[:, i], loc[:, i2]]   # (ne, nloc_lines)
                ok = (li[:, :, i] >= 0) & (li[:, :, i2] >= 0)
                np.add.at(ab, (li[:, :, i2][ok], w - (i2 - i), po[:, :, i2][ok]), vals[ok])
    return ab, w


class BlockLineSmoother:
    """B_s^-1 of Def. 3.2 with the literal line blocks: block Jacobi over the
    grid lines along axis s, each block R_L A P_L solved exactly."""

    def __init__(self, level: Level, s: int, A=None, Ae=None):
        self.level, self.s = level, s
        self.lin = line_nodes(level, s)
        ab, self.w = line_block_bands(level, s, A, Ae)
        self.factors = [sla.cholesky_banded(ab[k], lower=False) for k in range(len(ab))]

    def apply_inverse(self, res):
        r = np.asarray(res).ravel()
        out = np.zeros(self.level.N)
        for rows, c in zip(self.lin, self.factors):
            out[rows] = sla.cho_solve_banded((c, False), r[rows])
        return out.reshape(self.level.shape)

    def smooth(self, x, r, alpha):
        """x <- x + alpha B_s^-1 (r - A x)   (one step of Algorithm 2)."""
        return x + alpha * self.apply_inverse(r - self.level.apply(x))
