"""Bilinear (trilinear) finite-element matrix A~_p on the mesh of GLL nodes
(Sec. 3.1: the FEM line preconditioners replace A_p by A~_p).  Test
infrastructure only.

Reading of the unspecified construction: every cell between neighbouring
grid nodes is a Q1 element whose vertices are the physical node positions;
its stiffness is integrated with the 2-point Gauss-Legendre rule per axis
(exact for the affine case) under the isoparametric Q1 map.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .discretize import Level


def q1_stiffness(level: Level):
    """Sparse assembled A~ (no Dirichlet mask)."""
    d = level.dim
    shape = level.shape
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    corners = list(itertools.product((0, 1), repeat=d))   # in array-axis order (slowest first)
    # cell origins: all nodes except the last along each axis
    cell_shape = tuple(n - 1 for n in shape)
    origin = np.indices(cell_shape).reshape(d, -1)          # array-axis coordinates
    strides = np.cumprod((1,) + shape[::-1])[:-1][::-1]
    X = level.coords.reshape(d, -1)                          # physical coords per node (axis order x,y,z)
    nodes = np.stack([((origin + np.array(c)[:, None]) * strides[:, None]).sum(0) for c in corners], 1)
    Xc = X[:, nodes]                                         # (d_phys, ncell, 2^d)
    ncell = nodes.shape[0]
    Ke = np.zeros((ncell, len(corners), len(corners)))
    for qp in itertools.product(range(2), repeat=d):
        xq = np.array([g[i] for i in qp])                   # reference point, array-axis order
        # Q1 shape functions and reference gradients (array-axis order)
        N = np.array([np.prod([(1 + (2 * c[t] - 1) * xq[t]) / 2 for t in range(d)]) for c in corners])
        dN = np.zeros((len(corners), d))
        for k, c in enumerate(corners):
            for t in range(d):
                val = (2 * c[t] - 1) / 2
                for t2 in range(d):
                    if t2 != t:
                        val *= (1 + (2 * c[t2] - 1) * xq[t2]) / 2
                dN[k, t] = val
        # Jacobian Jm[cell, b, t] = d x_b / d r_t  (b physical, t array axis)
        Jm = np.einsum("bck,kt->cbt", Xc, dN)
        det = np.linalg.det(Jm)
        Jinv = np.linalg.inv(Jm)                             # [cell, t, b] = d r_t / d x_b
        grad = np.einsum("kt,ctb->ckb", dN, Jinv)            # d N_k / d x_b
        Ke += np.einsum("ckb,cjb,c->ckj", grad, grad, np.abs(det))
        del N
    rows = np.repeat(nodes[:, :, None], len(corners), axis=2)
    cols = np.repeat(nodes[:, None, :], len(corners), axis=1)
    A = sp.coo_matrix((Ke.ravel(), (rows.ravel(), cols.ravel())), shape=(level.N, level.N))
    return A.tocsr()


def line_band_from_matrix(level: Level, A, s: int):
    """(a, l, u) of the interior grid lines along axis s, read from an
    assembled sparse matrix (band 1 along the line)."""
    d = level.dim
    t = d - 1 - s
    shape = level.shape
    strides = np.cumprod((1,) + shape[::-1])[:-1][::-1]
    idx = np.arange(level.N).reshape(shape)
    inner = tuple(slice(1, -1) for _ in range(d))
    lin = np.moveaxis(idx[inner], t, -1)                     # (..., n)
    st = int(strides[t])
    diag = A.diagonal()
    a = diag[lin]
    up = np.asarray(A[lin.ravel(), lin.ravel() + st]).reshape(lin.shape)
    lo = np.asarray(A[lin.ravel(), lin.ravel() - st]).reshape(lin.shape)
    u = up.copy()
    l = lo.copy()
    u[..., -1] = 0.0
    l[..., 0] = 0.0
    return a, l, u
