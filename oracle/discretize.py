"""Discretisation on a structured grid of GLL spectral elements (Sec. 2.2-2.3).
Test infrastructure only.

Global nodal arrays have the grid shape (N_z, N_y, N_x) in 3-D or (N_y, N_x) in
2-D: lexicographic "left-right, bottom-top" order with x fastest (Fig. 4).
Element-local arrays have shape (E_z, E_y, E_x, p+1, p+1, p+1) (or the 2-D
analogue); local axis order matches the global one.  Physical axis a
(0 = x, 1 = y, 2 = z) is array axis dim-1-a.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import gll as _gll


def apply_1d(M, u, axis):
    """out[..., i, ...] = sum_k M[i, k] u[..., k, ...] along ``axis``: the
    one-dimensional factor of a tensor-product operator (sum factorisation)."""
    return np.moveaxis(np.tensordot(M, u, axes=([1], [axis])), 0, axis)


class Level:
    """One mesh level: element grid, GLL order p, nodal coordinates, and the
    quadrature-weighted geometry factors of eq. (discreteBilinear)."""

    def __init__(self, dim, nelem, p, coords):
        self.dim = int(dim)
        self.nelem = tuple(int(e) for e in nelem)
        self.p = int(p)
        self.shape = tuple(self.nelem[a] * p + 1 for a in reversed(range(dim)))
        self.N = int(np.prod(self.shape))
        self.coords = np.asarray(coords, dtype=np.float64).reshape((dim,) + self.shape)
        self.xi, self.rho = _gll.gll(p)
        self.D = _gll.derivative_matrix(self.xi)
        self._build_index()
        self._geometry()
        self.interior = np.zeros(self.shape, dtype=bool)
        self.interior[tuple(slice(1, -1) for _ in range(dim))] = True

    # ---- element <-> global ------------------------------------------------
    def eaxis(self, a):
        """Element-local array axis of physical axis a."""
        return self.dim + (self.dim - 1 - a)

    def _build_index(self):
        d, p = self.dim, self.p
        self.gidx = []
        for t in range(d):
            a = d - 1 - t
            base = np.arange(self.nelem[a])[:, None] * p + np.arange(p + 1)[None, :]
            shape = [1] * (2 * d)
            shape[t] = self.nelem[a]
            shape[d + t] = p + 1
            self.gidx.append(base.reshape(shape))
        self.gidx = tuple(self.gidx)
        strides = np.cumprod((1,) + self.shape[::-1])[:-1][::-1]
        lin = sum(self.gidx[t] * int(strides[t]) for t in range(d))
        self.eshape = tuple(self.nelem[::-1]) + (p + 1,) * d
        self.lin = np.broadcast_to(lin, self.eshape)

    def to_elements(self, u):
        return np.asarray(u).reshape(self.shape)[self.gidx]

    def from_elements(self, ue):
        """Direct stiffness summation: add element-local values at shared nodes."""
        y = np.bincount(self.lin.ravel(), weights=np.asarray(ue).ravel(), minlength=self.N)
        return y.reshape(self.shape)

    def local_weights(self):
        """prod_a rho[i_a] at every element-local node."""
        d = self.dim
        w = np.ones((1,) * d + (self.p + 1,) * d)
        for a in range(d):
            shape = [1] * (2 * d)
            shape[self.eaxis(a)] = self.p + 1
            w = w * self.rho.reshape(shape)
        return w

    # ---- geometry (isoparametric, Sec. 2.2) --------------------------------
    def _geometry(self):
        d = self.dim
        Xe = [self.to_elements(self.coords[b]) for b in range(d)]
        Jm = np.empty(self.eshape + (d, d))
        for b in range(d):
            for a in range(d):
                Jm[..., b, a] = apply_1d(self.D, Xe[b], self.eaxis(a))  # dx_b/dr_a
        det = np.linalg.det(Jm)
        if np.any(det <= 0):
            raise ValueError("non-positive Jacobian")
        Jinv = np.linalg.inv(Jm)  # Jinv[..., a, c] = dr_a/dx_c
        w = self.local_weights()
        self.det = det
        self.G = np.empty((d, d) + self.eshape)
        for a in range(d):
            for b in range(d):
                self.G[a, b] = w * det * np.sum(Jinv[..., a, :] * Jinv[..., b, :], axis=-1)
        self.mass_e = w * det

    def mass(self):
        """Diagonal of M: collocated GLL quadrature, M_ii = rho rho |J| summed
        over the elements sharing node i (reading of the garbled M formula)."""
        return self.from_elements(self.mass_e)

    # ---- operator ----------------------------------------------------------
    def apply_full(self, u):
        """A u without any Dirichlet mask: sum over elements of
        sum_ab D_a^T (G_ab (D_b u_e)), then summed at shared nodes."""
        d = self.dim
        ue = self.to_elements(u)
        grads = [apply_1d(self.D, ue, self.eaxis(a)) for a in range(d)]
        ye = np.zeros(self.eshape)
        for a in range(d):
            wa = sum(self.G[a, b] * grads[b] for b in range(d))
            ye += apply_1d(self.D.T, wa, self.eaxis(a))
        return self.from_elements(ye)

    def apply(self, u):
        """A restricted to interior unknowns: boundary entries of the input are
        ignored and boundary rows of the output are zero."""
        y = self.apply_full(np.where(self.interior, u, 0.0))
        return np.where(self.interior, y, 0.0)

    def element_matrices(self, sl=slice(None)):
        """Element stiffness matrices from the quadrature definition,
        A_e = sum_ab B_a^T diag(G_ab) B_b with B_a = derivative along axis a
        (Kronecker form), flattened in local lexicographic order."""
        d, n1 = self.dim, self.p + 1
        I = np.eye(n1)
        B = []
        for a in range(d):
            mats = [I] * d
            mats[d - 1 - a] = self.D
            K = mats[0]
            for m in mats[1:]:
                K = np.kron(K, m)
            B.append(K)
        eflat = self.G.reshape((d, d, -1, n1 ** d))[:, :, sl]
        ne = eflat.shape[2]
        Ae = np.zeros((ne, n1 ** d, n1 ** d))
        for a in range(d):
            for b in range(d):
                Ae += np.einsum("qi,eq,qj->eij", B[a], eflat[a, b], B[b], optimize=True)
        return Ae

    def assemble(self):
        """Sparse assembled A (no Dirichlet mask), from the element matrices."""
        n1d = (self.p + 1) ** self.dim
        Ae = self.element_matrices()
        lin = self.lin.reshape(-1, n1d)
        rows = np.repeat(lin[:, :, None], n1d, axis=2)
        cols = np.repeat(lin[:, None, :], n1d, axis=1)
        A = sp.coo_matrix((Ae.ravel(), (rows.ravel(), cols.ravel())), shape=(self.N, self.N))
        return A.tocsr()

    def interior_index(self):
        return np.flatnonzero(self.interior.ravel())


def lift(level: Level, f, g):
    """Dirichlet lifting (Sec. 2.3): v = g on the boundary and 0 inside,
    f0 = M f - A v on interior nodes (0 on the boundary).  Returns (f0, v);
    the solution is u = w + v with A w = f0."""
    v = np.where(level.interior, 0.0, np.asarray(g).reshape(level.shape))
    f0 = level.mass() * np.asarray(f).reshape(level.shape) - level.apply_full(v)
    return np.where(level.interior, f0, 0.0), v
