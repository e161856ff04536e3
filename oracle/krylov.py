"""Outer Krylov solvers.  Test infrastructure only.

The paper uses GMRES (Sec. 3) and stops at a residual reduction of 1e-8
(Sec. 4); the solver built here uses preconditioned CG.  Because the
gamma-cycle for gamma >= 2 is not a symmetric operator (pre- and
post-smoothing are adjoint only for one pass), the default is flexible CG
(Polak-Ribiere beta = z_{k+1}.(r_{k+1} - r_k) / z_k.r_k); plain PCG
(Fletcher-Reeves beta) is kept as an option.  Relative residual: Euclidean
norm over the interior unknowns, relative to the initial residual with x0 = 0.
"""
from __future__ import annotations

import numpy as np


def fcg(apply_A, apply_M, b, tol, maxit, flexible=True):
    """Returns (x, iterations, history); iterations = number of A products
    after which ||r|| <= tol ||r0|| (0 if b = 0)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.sqrt(np.vdot(r, r))
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = apply_M(r)
    p = z.copy()
    rz = np.vdot(r, z)
    for k in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / np.vdot(p, q)
        x = x + alpha * p
        r_new = r - alpha * q
        rel = np.sqrt(np.vdot(r_new, r_new)) / r0
        hist.append(rel)
        if rel <= tol:
            return x, k, hist
        z = apply_M(r_new)
        rz_new = np.vdot(r_new, z)
        beta = (rz_new - np.vdot(r, z)) / rz if flexible else rz_new / rz
        p = z + beta * p
        r, rz = r_new, rz_new
    return x, maxit, hist


def gmres(apply_A, apply_M, b, tol, maxit):
    """Right-preconditioned GMRES without restart, x0 = 0; stops when the
    least-squares residual estimate drops below tol ||b||.  Returns
    (x, iterations, history)."""
    b = np.asarray(b, dtype=np.float64)
    shape = b.shape
    bf = b.ravel()
    beta = np.linalg.norm(bf)
    hist = [1.0]
    if beta == 0.0:
        return np.zeros(shape), 0, hist
    V = [bf / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    k_done = maxit
    for k in range(maxit):
        z = np.asarray(apply_M(V[k].reshape(shape))).ravel()
        Z.append(z)
        w = np.asarray(apply_A(z.reshape(shape))).ravel()
        for i in range(k + 1):               # modified Gram-Schmidt
            H[i, k] = np.dot(w, V[i])
            w = w - H[i, k] * V[i]
        H[k + 1, k] = np.linalg.norm(w)
        V.append(w / H[k + 1, k] if H[k + 1, k] != 0 else w)
        for i in range(k):                   # apply previous rotations
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        rr = np.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = H[k, k] / rr, H[k + 1, k] / rr
        H[k, k] = rr
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        rel = abs(g[k + 1]) / beta
        hist.append(rel)
        if rel <= tol:
            k_done = k + 1
            break
    y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
    x = sum(y[i] * Z[i] for i in range(k_done))
    return x.reshape(shape), k_done, hist
