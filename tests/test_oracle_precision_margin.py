"""The precision the outer apply needs, measured on the oracle: flexible CG
whose operator products are rounded to k significant bits after every
multiply and add (a model of an apply carried in k-bit arithmetic) returns an
iterate whose true residual ||f0 - A w|| / ||f0||, computed in FP64, stays at
the recurrence residual the iteration reports for k = 48 (the float-float
format) down to tol = 1e-12, and parts from it for k = 32 (FP32-like).  This
is the margin behind serving mixed-precision solves with tol >= 1e-12 by a
float-float outer apply."""
import numpy as np
import pytest

from oracle import solve as osolve
from oracle.discretize import apply_1d, lift
from oracle.krylov import fcg
from paper_2504_10710_gb300 import inputs


def _round_bits(x, bits):
    """x rounded to `bits` significant bits (Veltkamp splitting of FP64)."""
    c = x * float(2 ** (53 - bits) + 1)
    return c - (c - x)


def _apply_rounded(fine, u, bits):
    """A u on interior rows, every product and partial sum of the
    sum-factorised element products rounded to `bits` bits."""
    r = lambda v: _round_bits(v, bits)
    u = np.where(fine.interior, u, 0.0)
    n1 = fine.p + 1
    ue, D, G = r(fine.to_elements(u)), r(fine.D), r(fine.G)

    def contract(M, v, axis):
        out = np.zeros_like(v)
        for i in range(n1):
            acc = 0.0
            for m in range(n1):
                acc = r(acc + r(M[i, m] * np.take(v, m, axis=axis)))
            idx = [slice(None)] * v.ndim
            idx[axis] = i
            out[tuple(idx)] = acc
        return out

    grads = [contract(D, ue, fine.eaxis(a)) for a in range(fine.dim)]
    ye = np.zeros(fine.eshape)
    for a in range(fine.dim):
        wa = 0.0
        for b in range(fine.dim):
            wa = r(wa + r(G[a, b] * grads[b]))
        ye = r(ye + contract(D.T, wa, fine.eaxis(a)))
    return np.where(fine.interior, fine.from_elements(ye), 0.0)


@pytest.fixture(scope="module")
def setup():
    wl = inputs.random2d((12, 12), 8, amp=0.1, seed=71)
    fine, hier = osolve.build(wl, smoother="gll", restriction="transpose")
    f0, _ = lift(fine, wl.sample_rhs(fine.coords)[0], wl.sample_dirichlet(fine.coords))
    M = lambda r: hier.precondition(r, 1, 2.0 / 3.0, 1)
    return fine, f0, M


def _true_and_reported(setup, bits, tol):
    fine, f0, M = setup
    w, _, hist = fcg(lambda u: _apply_rounded(fine, u, bits), M, f0, tol, 80)
    true = np.linalg.norm(f0 - fine.apply(w)) / np.linalg.norm(f0)
    return true, hist[-1]


def test_rounding_model_is_exact_at_53_bits(setup):
    fine, f0, _ = setup
    rng = np.random.default_rng(3)
    u = np.where(fine.interior, rng.standard_normal(fine.shape), 0.0)
    a, b = _apply_rounded(fine, u, 53), fine.apply(u)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
def test_48_bit_apply_keeps_the_true_residual(setup, tol):
    true, reported = _true_and_reported(setup, 48, tol)
    assert reported <= tol
    assert true <= 1.5 * tol, (true, reported)


def test_32_bit_apply_loses_the_true_residual(setup):
    """The check has teeth: with FP32-like products the true residual stalls
    far above a 1e-12 recurrence residual."""
    true, reported = _true_and_reported(setup, 32, 1e-12)
    assert reported <= 1e-12
    assert true > 100 * 1e-12, (true, reported)
