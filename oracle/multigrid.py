"""p-multigrid hierarchy and the gamma-cycle (Sec. 3.3, Def. 3.12, Algorithm 2).
Test infrastructure only.

Readings taken where the paper is silent or ambiguous:
  * Order chain: p_{l-1} = floor(p_l / 2) (coarsening factor f = 2 of
    Prop. 3.13).  The chain stops at the lowest order whose grid has interior
    unknowns: p = 1 when every axis has at least two elements, p = 2
    otherwise (one element along an axis has no interior node there at p = 1;
    a single element is the paper's case).
  * Coarse geometry: coarse nodes are the fine element's coordinate polynomial
    evaluated at the coarse GLL points, and A_l is rediscretised on that mesh
    with eq. (discreteBilinear) (the paper rediscretises and notes that the
    coarse levels only approximate the geometry).
  * Transfers: P_l interpolates a degree-p_{l-1} field to the GLL(p_l) nodes of
    the same elements (a tensor product of 1-D global interpolations on the
    structured grid).  The paper defines both R_l and P_l as "interpolation
    operators from one basis to another, at the corresponding quadrature nodes"
    and in the same paragraph writes R_l = P_l^T.  Both are provided:
    restriction="interp" evaluates the fine nodal field at the coarse GLL nodes
    (the reading under which Table 1 is reproduced to within one iteration),
    restriction="transpose" applies P_l^T.  Dirichlet rows of the coarse
    residual are zero in both.
  * Algorithm 2 as printed restarts every pass of the gamma loop from x_{2m};
    the passes are chained instead (each pass starts from the previous y_{2m}),
    which matches the per-visit cost (gamma + 1) smoothings used in the proof
    of Prop. 3.13.
  * Smoother order: pre-smoothing along x then y (then z in 3-D);
    post-smoothing in the reverse order, as in Algorithm 2 for 2-D.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import gll as _gll
from .discretize import Level, apply_1d
from .fem import line_band_from_matrix, q1_stiffness
from .lines import BlockLineSmoother, LineSmoother


def order_chain(p_fine: int, multi_element: bool):
    p0 = 1 if multi_element else 2
    chain = [p_fine]
    while chain[-1] > p0:
        nxt = chain[-1] // 2
        if nxt < p0:
            nxt = p0
        chain.append(nxt)
    return chain


def coarse_coords(level: Level, p_c: int):
    """Nodal coordinates of the GLL(p_c) mesh: the fine coordinate polynomial
    of every element evaluated at the coarse GLL points."""
    d, p_f = level.dim, level.p
    J = _gll.interpolation_matrix(p_f, p_c)     # J[i_c, k_f]
    shape_c = tuple(level.nelem[a] * p_c + 1 for a in reversed(range(d)))
    out = np.zeros((d,) + shape_c)
    for b in range(d):
        xe = level.to_elements(level.coords[b])
        for a in range(d):
            xe = apply_1d(J, xe, level.eaxis(a))
        # write element-local values into the global coarse grid (shared nodes
        # receive identical values: the trace on a face depends on face nodes only)
        idx = []
        for t in range(d):
            a = d - 1 - t
            base = np.arange(level.nelem[a])[:, None] * p_c + np.arange(p_c + 1)[None, :]
            shp = [1] * (2 * d)
            shp[t] = level.nelem[a]
            shp[d + t] = p_c + 1
            idx.append(np.broadcast_to(base.reshape(shp), xe.shape))
        out[b][tuple(idx)] = xe
    return out


def interp_1d_global(nelem: int, p_c: int, p_f: int):
    """Global 1-D interpolation matrix (nelem p_f + 1) x (nelem p_c + 1) from a
    continuous piecewise degree-p_c field to the GLL(p_f) nodes."""
    J = _gll.interpolation_matrix(p_c, p_f)     # J[i_f, k_c]
    P = np.zeros((nelem * p_f + 1, nelem * p_c + 1))
    for e in range(nelem):
        P[e * p_f:(e + 1) * p_f + 1, e * p_c:(e + 1) * p_c + 1] = J
    return P


class Hierarchy:
    """Levels l = L (finest) ... 0 (coarsest), with smoothers, transfers and
    the exact coarsest solver M_0^-1 = A_0^-1."""

    def __init__(self, fine: Level, chain=None, smoother="gll", restriction="interp"):
        multi = all(e > 1 for e in fine.nelem)       # p = 1 has interior unknowns
        self.chain = chain or order_chain(fine.p, multi)
        self.levels = [fine]
        for p_c in self.chain[1:]:
            prev = self.levels[-1]
            self.levels.append(Level(fine.dim, fine.nelem, p_c, coarse_coords(prev, p_c)))
        self.levels = self.levels[::-1]        # index 0 = coarsest
        self.L = len(self.levels) - 1
        d = fine.dim
        self.smoother = smoother
        self.smoothers = [None] + [self._make_smoothers(lv) for lv in self.levels[1:]]
        # P1D[l][a]: interpolation from level l-1 to level l along axis a
        self.P1D = [None] + [
            [interp_1d_global(fine.nelem[a], self.levels[l - 1].p, self.levels[l].p) for a in range(d)]
            for l in range(1, self.L + 1)]
        # R1D[l][a]: restriction from level l to level l-1 along axis a
        if restriction == "interp":
            self.R1D = [None] + [
                [interp_1d_global(fine.nelem[a], self.levels[l].p, self.levels[l - 1].p) for a in range(d)]
                for l in range(1, self.L + 1)]
        elif restriction == "transpose":
            self.R1D = [None] + [[P.T for P in self.P1D[l]] for l in range(1, self.L + 1)]
        else:
            raise ValueError(restriction)
        self.restriction = restriction
        lv0 = self.levels[0]
        A0 = lv0.assemble()
        ii = lv0.interior_index()
        self.coarse_index = ii
        self.coarse_factor = sla.cho_factor(A0[ii][:, ii].toarray())

    def _make_smoothers(self, lv):
        """Line smoothers of one level.  "gll": Def. 3.2's R A_p P line blocks;
        "gll_band1": their band-1 part; "fem": R A~_p P (tridiagonal)."""
        d = lv.dim
        if self.smoother == "gll":
            n1d = (lv.p + 1) ** d
            Ae = lv.element_matrices() if int(np.prod(lv.nelem)) * n1d * n1d <= 5e7 else None
            return [BlockLineSmoother(lv, s, Ae=Ae) for s in range(d)]
        if self.smoother == "gll_band1":
            return [LineSmoother(lv, s) for s in range(d)]
        if self.smoother == "fem":
            At = q1_stiffness(lv)
            return [LineSmoother(lv, s, line_band_from_matrix(lv, At, s)) for s in range(d)]
        raise ValueError(self.smoother)

    def prolong(self, l, e):
        """P_l e: tensor product of the 1-D interpolations."""
        d = self.levels[l].dim
        x = np.asarray(e)
        for a in range(d):
            x = apply_1d(self.P1D[l][a], x, d - 1 - a)
        return x

    def restrict(self, l, r):
        """R_l r (tensor product of the 1-D restrictions), with the coarse
        Dirichlet rows set to zero."""
        d = self.levels[l].dim
        x = np.asarray(r)
        for a in range(d):
            x = apply_1d(self.R1D[l][a], x, d - 1 - a)
        return np.where(self.levels[l - 1].interior, x, 0.0)

    def coarse_solve(self, r):
        lv0 = self.levels[0]
        out = np.zeros(lv0.N)
        out[self.coarse_index] = sla.cho_solve(self.coarse_factor, np.asarray(r).ravel()[self.coarse_index])
        return out.reshape(lv0.shape)

    def cycle(self, l, r, gamma, alpha, m=1, trace=None):
        """Action M_l^-1 r of the gamma-cycle (Algorithm 2), starting from x0 = 0."""
        if l == 0:
            if trace is not None:
                trace.append(("coarse", 0))
            return self.coarse_solve(r)
        lv = self.levels[l]
        sm = self.smoothers[l]
        d = lv.dim
        x = np.zeros(lv.shape)
        for s in range(d):                      # pre: x, then y (then z)
            for _ in range(m):
                if trace is not None:
                    trace.append(("smooth", l, s))
                x = sm[s].smooth(x, r, alpha)
        for _ in range(gamma):
            rc = self.restrict(l, r - lv.apply(x))
            x = x + self.prolong(l, self.cycle(l - 1, rc, gamma, alpha, m, trace))
            for s in reversed(range(d)):        # post: reverse order
                for _ in range(m):
                    if trace is not None:
                        trace.append(("smooth", l, s))
                    x = sm[s].smooth(x, r, alpha)
        return x

    def precondition(self, r, gamma, alpha, m=1, trace=None):
        return self.cycle(self.L, np.asarray(r).reshape(self.levels[self.L].shape), gamma, alpha, m, trace)
