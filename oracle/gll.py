"""GLL quadrature (Def. 2.1), Lagrange basis derivative (Def. 2.2) and
interpolation between GLL orders (Sec. 3.3).  Test infrastructure only."""
from __future__ import annotations

import numpy as np


def legendre(p: int, x):
    """L_p(x) and L_p'(x) by the three-term recurrence
    (n+1) L_{n+1} = (2n+1) x L_n - n L_{n-1}, and the derivative from
    L_p' = p (L_{p-1} - x L_p) / (1 - x^2) away from +-1 (at +-1 the closed
    value L_p'(+-1) = (+-1)^{p-1} p (p+1) / 2)."""
    x = np.asarray(x, dtype=np.float64)
    Lm, L = np.ones_like(x), x.copy()
    if p == 0:
        return Lm, np.zeros_like(x)
    for n in range(1, p):
        Lm, L = L, ((2 * n + 1) * x * L - n * Lm) / (n + 1)
    # now L = L_p, Lm = L_{p-1}
    with np.errstate(divide="ignore", invalid="ignore"):
        dL = p * (Lm - x * L) / (1.0 - x * x)
    end = np.abs(np.abs(x) - 1.0) < 1e-15
    dL = np.where(end, np.sign(x) ** (p - 1) * p * (p + 1) / 2.0, dL)
    return L, dL


def gll(p: int):
    """Nodes xi_0 = -1 < ... < xi_p = 1 with L_p'(xi_n) = 0 inside, and weights
    rho_n = 2 / (p (p+1) L_p(xi_n)^2)   (Def. 2.1).

    Interior nodes: Newton's method on L_p', started from the
    Chebyshev-Gauss-Lobatto points -cos(pi n / p); the second derivative comes
    from Legendre's equation (1 - x^2) L'' = 2 x L' - p (p+1) L."""
    if p < 1:
        raise ValueError("GLL order must be >= 1")
    xi = -np.cos(np.pi * np.arange(p + 1) / p)
    inner = xi[1:-1].copy()
    for _ in range(100):
        L, dL = legendre(p, inner)
        d2L = (2 * inner * dL - p * (p + 1) * L) / (1 - inner * inner)
        step = dL / d2L
        inner -= step
        if np.all(np.abs(step) < 1e-16):
            break
    xi[1:-1] = inner
    xi[0], xi[-1] = -1.0, 1.0
    L, _ = legendre(p, xi)
    rho = 2.0 / (p * (p + 1) * L * L)
    return xi, rho


def barycentric_weights(nodes):
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    w = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                w[j] /= nodes[j] - nodes[k]
    return w


def derivative_matrix(nodes):
    """D[i, j] = pi_j'(xi_i) for the Lagrange basis on ``nodes`` (Def. 2.2).

    Off-diagonal entries from differentiating the Lagrange polynomial in
    barycentric form, pi_j'(xi_i) = (w_j / w_i) / (xi_i - xi_j); the diagonal
    from sum_j pi_j = 1, i.e. each row sums to zero."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    w = barycentric_weights(nodes)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (nodes[i] - nodes[j])
        D[i, i] = -D[i].sum()
    return D


def lagrange_eval(nodes, x):
    """Matrix V[i, k] = pi_k(x_i) for the Lagrange basis on ``nodes``,
    straight from the product definition (Def. 2.2)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    V = np.ones((len(x), len(nodes)))
    for k in range(len(nodes)):
        for m in range(len(nodes)):
            if m != k:
                V[:, k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
    return V


def interpolation_matrix(p_from: int, p_to: int):
    """J[i, k] = pi_k^{(p_from)}(xi_i^{(p_to)}): values at GLL(p_to) nodes of the
    degree-p_from interpolant (Sec. 3.3, P_l = interpolation between bases)."""
    return lagrange_eval(gll(p_from)[0], gll(p_to)[0])
