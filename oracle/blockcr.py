"""Block cyclic reduction as a direct multigrid (Thm. 3.8 with blocks of size
m > 1, Prop. 3.7, Cor. 3.9), used as the exact solver of the coarsest level.
Test infrastructure only: nothing in the library imports this module.

Notation of Def. 3.5: a block-tridiagonal matrix M with diagonal blocks A_i,
sub-diagonal blocks L_i (row i, column i - 1) and super-diagonal blocks U_i
(row i, column i + 1), i = 1..n (1-based; L_1 = U_n = 0).  With 1-based
indices the odd blocks are the fine points and the even blocks the coarse
points.  One level is Algorithm 1 with the operators of Thm. 3.8:
  x = S^-1 g            S^-1 = blockdiag(A_1^-1, 0, A_3^-1, 0, ...)
  c = R (g - M x)       R = P^T
  e = M_0^-1 c          M_0 = D - C A^-1 B, block-tridiagonal (Prop. 3.7)
  y = x + P e           P: identity on even blocks; odd block j takes
                        -A_j^-1 L_j from coarse j - 1 and -A_j^-1 U_j from j + 1
The coarse stencil of Prop. 3.7 for even i, with the diagonal read from the
explicit product C A^-1 B (the printed diagonal repeats the sub-diagonal's
L_{i-1}; the product gives U_{i-1}):
  L'_i = -L_i A_{i-1}^-1 L_{i-1}
  A'_i = A_i - L_i A_{i-1}^-1 U_{i-1} - U_i A_{i+1}^-1 L_{i+1}
  U'_i = -U_i A_{i+1}^-1 U_{i+1}
Cor. 3.9 applies the step recursively to M_0.  `levels` bounds the
recursion: after that many levels the remaining coarse system is solved by a
dense direct solve (levels=None recurses until one block is left).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def blocks_of(M, nb: int, m: int):
    """Blocks (A, L, U) of a dense block-tridiagonal matrix of nb blocks of
    size m (Def. 3.5): arrays of shape (nb, m, m), L[0] = U[-1] = 0."""
    M = np.asarray(M, dtype=float)
    assert M.shape == (nb * m, nb * m)
    A = np.zeros((nb, m, m))
    L = np.zeros((nb, m, m))
    U = np.zeros((nb, m, m))
    for i in range(nb):
        s = slice(i * m, (i + 1) * m)
        A[i] = M[s, s]
        if i > 0:
            L[i] = M[s, slice((i - 1) * m, i * m)]
        if i + 1 < nb:
            U[i] = M[s, slice((i + 1) * m, (i + 2) * m)]
    return A, L, U


def assemble(A, L, U):
    """Dense matrix of the block-tridiagonal (A, L, U)."""
    nb, m, _ = A.shape
    M = np.zeros((nb * m, nb * m))
    for i in range(nb):
        s = slice(i * m, (i + 1) * m)
        M[s, s] = A[i]
        if i > 0:
            M[s, slice((i - 1) * m, i * m)] = L[i]
        if i + 1 < nb:
            M[s, slice((i + 1) * m, (i + 2) * m)] = U[i]
    return M


def two_level_operators(A, L, U):
    """Dense S^-1, P, R = P^T and the blocks of M_0 of Thm. 3.8 / Prop. 3.7
    for one level (odd blocks = 0-based indices 0, 2, 4, ...)."""
    nb, m, _ = A.shape
    odd = list(range(0, nb, 2))
    even = list(range(1, nb, 2))
    Ainv = {j: np.linalg.inv(A[j]) for j in odd}
    Sinv = np.zeros((nb * m, nb * m))
    for j in odd:
        Sinv[j * m:(j + 1) * m, j * m:(j + 1) * m] = Ainv[j]
    nc = len(even)
    P = np.zeros((nb * m, nc * m))
    for k, i in enumerate(even):
        P[i * m:(i + 1) * m, k * m:(k + 1) * m] = np.eye(m)
        j = i - 1                                    # odd block left of coarse i
        P[j * m:(j + 1) * m, k * m:(k + 1) * m] = -Ainv[j] @ U[j]
        j = i + 1                                    # odd block right of coarse i
        if j < nb:
            P[j * m:(j + 1) * m, k * m:(k + 1) * m] = -Ainv[j] @ L[j]
    R = P.T
    A0 = np.zeros((nc, m, m))
    L0 = np.zeros((nc, m, m))
    U0 = np.zeros((nc, m, m))
    for k, i in enumerate(even):
        A0[k] = A[i] - L[i] @ Ainv[i - 1] @ U[i - 1]
        L0[k] = -L[i] @ Ainv[i - 1] @ L[i - 1] if k > 0 else 0.0
        if i + 1 < nb:
            A0[k] -= U[i] @ Ainv[i + 1] @ L[i + 1]
            if k + 1 < nc:
                U0[k] = -U[i] @ Ainv[i + 1] @ U[i + 1]
    return Sinv, P, R, (A0, L0, U0)


def block_cr_solve(A, L, U, g, levels=None):
    """Solve M x = g (g of shape (nb, m) or (nb * m,)) by Algorithm 1 applied
    recursively (Cor. 3.9); `levels` CR levels, then a dense direct solve of
    the remaining coarse system (Cholesky: the coarse systems of an SPD M are
    SPD Schur complements)."""
    nb, m, _ = A.shape
    g = np.asarray(g, dtype=float).reshape(nb * m)
    if nb == 1 or levels == 0:
        M = assemble(A, L, U)
        return sla.cho_solve(sla.cho_factor(M), g)
    M = assemble(A, L, U)
    Sinv, P, R, (A0, L0, U0) = two_level_operators(A, L, U)
    x = Sinv @ g                                     # x = S^-1 g
    c = R @ (g - M @ x)                              # c = R (g - M x)
    e = block_cr_solve(A0, L0, U0, c, None if levels is None else levels - 1)
    return x + P @ e                                 # y = x + P e


def grid_blocks(M, shape):
    """Block partition of a lexicographically numbered grid operator (x
    fastest): block i is the i-th index of the slowest axis (a grid line in
    2-D, a plane in 3-D).  shape: interior points per axis, slowest last
    (nx, ny) or (nx, ny, nz).  Returns (A, L, U, nb, m)."""
    nb = int(shape[-1])
    m = int(np.prod(shape[:-1]))
    A, L, U = blocks_of(M, nb, m)
    return A, L, U, nb, m
