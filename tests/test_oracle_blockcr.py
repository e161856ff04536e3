"""Pins of the block cyclic-reduction oracle (Thm. 3.8 with m > 1, Prop. 3.7,
Cor. 3.9) against the library dense solve, the independent scalar CR oracle
(m = 1), the explicit Schur complement of the odd-even reordered matrix, and
the one-step exactness that Thm. 3.8 states."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import blockcr
from oracle.discretize import Level
from oracle.gll import gll
from oracle.lines import cr_solve
from oracle.multigrid import Hierarchy
from paper_2504_10710_gb300 import inputs


def _random_spd_blocks(nb, m, seed):
    """Random symmetric block-tridiagonal matrix, made SPD by a diagonal shift."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nb, m, m))
    A = A + np.transpose(A, (0, 2, 1))
    L = np.zeros((nb, m, m))
    U = np.zeros((nb, m, m))
    for i in range(1, nb):
        L[i] = rng.standard_normal((m, m))
        U[i - 1] = L[i].T
    M = blockcr.assemble(A, L, U)
    shift = -np.linalg.eigvalsh(M).min() + 1.0
    A = A + shift * np.eye(m)[None]
    return A, L, U


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 7, 8, 15, 16, 17])
@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_block_cr_equals_dense_solve(nb, m):
    A, L, U = _random_spd_blocks(nb, m, 100 * nb + m)
    M = blockcr.assemble(A, L, U)
    g = np.random.default_rng(nb + 7 * m).standard_normal(nb * m)
    ref = np.linalg.solve(M, g)
    maxlev = int(np.ceil(np.log2(nb + 1)))
    for levels in [None] + list(range(0, maxlev + 1)):
        x = blockcr.block_cr_solve(A, L, U, g, levels)
        np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10 * np.abs(ref).max(), err_msg=str(levels))


@pytest.mark.parametrize("nb", [1, 2, 6, 15, 31, 40])
def test_scalar_blocks_reduce_to_scalar_cr(nb):
    """m = 1: the block recursion is the scalar CR of Cor. 3.9 (an independent
    vectorised implementation)."""
    rng = np.random.default_rng(nb)
    a = 4.0 + rng.random(nb)
    o = -rng.random(nb - 1) if nb > 1 else np.zeros(0)
    l = np.concatenate([[0.0], o])
    u = np.concatenate([o, [0.0]])
    g = rng.standard_normal(nb)
    A = a.reshape(nb, 1, 1)
    L = l.reshape(nb, 1, 1)
    U = u.reshape(nb, 1, 1)
    np.testing.assert_allclose(blockcr.block_cr_solve(A, L, U, g), cr_solve(a, l, u, g), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("nb,m", [(5, 3), (8, 2), (9, 4)])
def test_coarse_blocks_are_the_schur_complement(nb, m):
    """Prop. 3.7: M_0 = D - C A^-1 B of Q^T M Q, block by block.  The printed
    diagonal (with L_{i-1} in place of U_{i-1}) fails this test."""
    A, L, U = _random_spd_blocks(nb, m, 7 * nb + m)
    M = blockcr.assemble(A, L, U)
    odd = np.concatenate([np.arange(j * m, (j + 1) * m) for j in range(0, nb, 2)])
    even = np.concatenate([np.arange(i * m, (i + 1) * m) for i in range(1, nb, 2)])
    S = M[np.ix_(even, even)] - M[np.ix_(even, odd)] @ np.linalg.solve(M[np.ix_(odd, odd)], M[np.ix_(odd, even)])
    _, _, _, (A0, L0, U0) = blockcr.two_level_operators(A, L, U)
    np.testing.assert_allclose(blockcr.assemble(A0, L0, U0), S, rtol=0, atol=1e-11 * np.abs(S).max())
    printed = A[1] - L[1] @ np.linalg.inv(A[0]) @ L[0] - U[1] @ np.linalg.inv(A[2]) @ L[2]
    assert np.abs(printed - S[:m, :m]).max() > 1e-3 * np.abs(S).max()


@pytest.mark.parametrize("nb,m", [(7, 2), (10, 3)])
def test_two_level_method_is_exact_in_one_step(nb, m):
    """Thm. 3.8: with M_0 solved exactly, the two-level preconditioner
    B = S^-1 + P M_0^-1 R (I - M S^-1) of Algorithm 1 satisfies B M = I."""
    A, L, U = _random_spd_blocks(nb, m, 3 * nb + m)
    M = blockcr.assemble(A, L, U)
    Sinv, P, R, (A0, L0, U0) = blockcr.two_level_operators(A, L, U)
    M0 = blockcr.assemble(A0, L0, U0)
    np.testing.assert_allclose(R @ M @ P, M0, atol=1e-10 * np.abs(M0).max())   # Galerkin coarse operator
    B = Sinv + P @ np.linalg.solve(M0, R @ (np.eye(nb * m) - M @ Sinv))
    np.testing.assert_allclose(B @ M, np.eye(nb * m), atol=1e-10)


@pytest.mark.parametrize("wl", [inputs.random2d((8, 6), 2, amp=0.15, seed=3),
                                inputs.random3d((4, 3, 4), 2, amp=0.15, seed=4)], ids=["2d", "3d"])
def test_block_cr_on_the_coarsest_grid_operator(wl):
    """The coarsest level's operator, blocked by grid lines (2-D) or planes
    (3-D) of the slowest axis, solved at every CR depth."""
    coords = wl.coords(gll(wl.order)[0])
    hier = Hierarchy(Level(wl.dim, wl.nelem, wl.order, coords), restriction="transpose")
    lv0 = hier.levels[0]
    ii = lv0.interior_index()
    M = lv0.assemble()[ii][:, ii].toarray()
    shape = tuple(n - 2 for n in lv0.shape[::-1])          # interior points, x first
    A, L, U, nb, m = blockcr.grid_blocks(M, shape)
    assert np.abs(blockcr.assemble(A, L, U) - M).max() == 0.0   # nothing outside the block band
    g = np.random.default_rng(5).standard_normal(nb * m)
    ref = sla.cho_solve(sla.cho_factor(M), g)
    for levels in range(0, int(np.ceil(np.log2(nb + 1))) + 1):
        x = blockcr.block_cr_solve(A, L, U, g, levels)
        np.testing.assert_allclose(x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
