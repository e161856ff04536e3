"""Pins for the oracle's GLL tables (Def. 2.1, Def. 2.2, Sec. 3.3 transfers)."""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import gll

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _num(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def test_closed_forms_small_orders():
    data = json.load(open(os.path.join(GOLD, "gll_closed_forms.json")))
    for p in ("1", "2", "3", "4"):
        xi, rho = gll.gll(int(p))
        np.testing.assert_allclose(xi, [_num(s) for s in data[p]["nodes"]], atol=1e-15)
        np.testing.assert_allclose(rho, [_num(s) for s in data[p]["weights"]], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 25))
def test_nodes_match_library_roots_of_Lp_derivative(p):
    xi, _ = gll.gll(p)
    if p >= 2:
        c = np.zeros(p + 1)
        c[p] = 1.0
        roots = np.sort(npleg.legroots(npleg.legder(c)))
        np.testing.assert_allclose(xi[1:-1], roots, atol=1e-13)
    assert xi[0] == -1.0 and xi[-1] == 1.0
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 25))
def test_quadrature_exactness_degree_2p_minus_1(p):
    xi, rho = gll.gll(p)
    assert abs(rho.sum() - 2.0) < 1e-13
    for k in range(0, 2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(rho, xi ** k) - exact) < 1e-12, (p, k)
    # first degree the rule misses: the Lobatto remainder for f = x^{2p},
    # exact - rule = -(p+1) p^3 2^{2p+1} ((p-1)!)^4 / ((2p+1) ((2p)!)^2)
    k = 2 * p
    rem = -((p + 1) * p ** 3 * 2 ** (2 * p + 1) * math.factorial(p - 1) ** 4
            / ((2 * p + 1) * math.factorial(2 * p) ** 2))
    err = 2.0 / (k + 1) - np.dot(rho, xi ** k)
    assert abs(err - rem) < 1e-13 + 1e-9 * abs(rem)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 12, 16])
def test_derivative_matrix_exact_on_polynomials(p):
    xi, _ = gll.gll(p)
    D = gll.derivative_matrix(xi)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-11 * p * p)
    for k in range(0, p + 1):
        np.testing.assert_allclose(D @ xi ** k, k * xi ** max(k - 1, 0) if k else 0 * xi,
                                   atol=1e-11 * p ** 2)


@pytest.mark.parametrize("p", [2, 3, 5, 8, 12])
def test_derivative_matrix_matches_legendre_closed_form(p):
    """Independent closed form (Deville-Fischer-Mund (2.4.9)):
    D_ij = L_p(x_i) / (L_p(x_j) (x_i - x_j)), D_00 = -p(p+1)/4, D_pp = p(p+1)/4."""
    xi, _ = gll.gll(p)
    c = np.zeros(p + 1)
    c[p] = 1.0
    L = npleg.legval(xi, c)
    ref = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            if i != j:
                ref[i, j] = L[i] / (L[j] * (xi[i] - xi[j]))
    ref[0, 0] = -p * (p + 1) / 4
    ref[p, p] = p * (p + 1) / 4
    np.testing.assert_allclose(gll.derivative_matrix(xi), ref, atol=1e-11 * p ** 2)


@pytest.mark.parametrize("p", range(1, 17))
def test_derivative_matrix_centro_antisymmetric(p):
    """GLL nodes are symmetric about 0 (x_{p-i} = -x_i), so l_{p-j}(x) = l_j(-x)
    and D_{p-i, p-j} = -D_ij; the 3-D apply's even-odd sweeps rely on it.
    With the even and odd halves of u, D u is recovered from half-size
    products: (Du)_i = A_i + B_i, (Du)_{p-i} = B_i - A_i."""
    xi, _ = gll.gll(p)
    np.testing.assert_allclose(xi[::-1], -xi, atol=1e-15)
    D = gll.derivative_matrix(xi)
    n, h = p + 1, (p + 1) // 2
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-12 * p * p)
    u = np.random.default_rng(p).standard_normal(n)
    for M in (D, D.T):
        ue = u[:h] + u[::-1][:h]
        uo = u[:h] - u[::-1][:h]
        E = 0.5 * (M[:h, :h] + M[:h, ::-1][:, :h])
        O = 0.5 * (M[:h, :h] - M[:h, ::-1][:, :h])
        A = E @ ue + (M[:h, h] * u[h] if n % 2 else 0.0)
        B = O @ uo
        out = np.empty(n)
        out[:h] = A + B
        out[::-1][:h] = B - A
        if n % 2:
            out[h] = M[h, :h] @ uo
        np.testing.assert_allclose(out, M @ u, atol=1e-12 * p * p * np.abs(u).max())


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (3, 7), (4, 8), (6, 12), (5, 11)])
def test_interpolation_exact_up_to_coarse_degree(pc, pf):
    J = gll.interpolation_matrix(pc, pf)
    xc, _ = gll.gll(pc)
    xf, _ = gll.gll(pf)
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-13)
    for k in range(pc + 1):
        np.testing.assert_allclose(J @ xc ** k, xf ** k, atol=1e-12)
    # endpoints are shared nodes: unit rows
    np.testing.assert_array_equal(J[0], np.eye(pc + 1)[0])
    np.testing.assert_array_equal(J[-1], np.eye(pc + 1)[-1])
