"""The 3-D stiffness apply at every specialised order against the oracle's
A_l x (eq. discreteBilinear), through the three kernels that serve 3-D:
the even-odd line kernel (FP32 p >= 4, FP64 p = 6, 7), the column kernel
(FP32 p <= 3) and the node-per-thread kernel (FP64 elsewhere).  A small
ragged grid runs one element per CTA; the 17 x 16 x 14 grid (3,808
elements) makes the even-odd kernel put three elements in a CTA with a
partial last CTA.  Tolerances as the parity tests: 1e-12 (FP64) and 5e-5
(FP32) relative to the largest entry."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.discretize import Level  # noqa: E402
from paper_2504_10710_gb300 import glls, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _check(nelem, p, seed):
    wl = inputs.random3d(nelem, p, amp=0.15, seed=seed)
    xi, _ = glls.gll(p)
    coords = wl.coords(xi)
    prob = glls.Problem(3, wl.nelem, p, coords)
    L = prob.levels - 1
    assert prob.info.order[L] == p
    lv = Level(3, wl.nelem, p, coords)
    x = np.where(lv.interior, inputs.random_field(lv.shape, seed + 100), 0.0)
    ref = lv.apply(x)
    scale = np.abs(ref).max()
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 5e-5)):
        y = torch.zeros(lv.N, dtype=dtype, device="cuda")
        prob.apply(L, torch.tensor(x.ravel(), dtype=dtype, device="cuda"), y)
        torch.cuda.synchronize()
        err = np.abs(y.double().cpu().numpy().reshape(lv.shape) - ref).max() / scale
        assert err < tol, (nelem, p, dtype, err)
    prob.close()


@pytest.mark.parametrize("p", range(1, 9))
def test_apply_every_order_small_grid(p):
    _check((3, 2, 2), p, 60 + p)


@pytest.mark.parametrize("p", range(4, 9))
def test_apply_several_elements_per_cta(p):
    _check((17, 16, 14), p, 70 + p)
