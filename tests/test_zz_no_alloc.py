"""The allocation-free restriction entry point.

glls_restrict_noalloc_f32 serves callers that cannot call cudaMalloc (for
instance code running under an allocator that owns all device memory, or a
path that must not pay cudaMalloc's implicit synchronisation): it keeps its
scratch in one fixed device array inside the library instead of the
problem's own buffers.  It
must give the same coarse residual as glls_restrict_f32, call after call,
and refuse levels larger than its fixed scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_10710_gb300 import glls, inputs  # noqa: E402

TOL32 = 5e-4   # the FP32 tolerance of the restriction parity tests (5e-5 x 10)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _interior(shape, seed):
    v = inputs.random_field(shape, seed)
    inner = np.zeros(shape, dtype=bool)
    inner[tuple(slice(1, -1) for _ in shape)] = True
    return torch.tensor(np.where(inner, v, 0.0).ravel(), dtype=torch.float32, device="cuda")


def _noalloc(prob, level, r, x, rc):
    fn = glls.lib().glls_restrict_noalloc_f32
    return fn(prob.h, level, C.c_void_p(r.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(rc.data_ptr()), None)


@pytest.mark.parametrize("wl", [inputs.random2d((6, 5), 8, amp=0.1, seed=3),
                                inputs.random3d((3, 2, 2), 5, amp=0.1, seed=4)], ids=["2d", "3d"])
def test_noalloc_restriction_matches_allocating_entry_point(wl):
    prob, _ = glls.problem_for(wl)
    for level in range(prob.levels - 1, 0, -1):
        shf, shc = prob.level_shape(level), prob.level_shape(level - 1)
        for call in range(2):          # two calls in a row share the scratch array
            r = _interior(shf, 100 + 10 * level + call)
            x = _interior(shf, 200 + 10 * level + call)
            ref = torch.zeros(int(np.prod(shc)), dtype=torch.float32, device="cuda")
            out = torch.full_like(ref, 7.0)
            prob.restrict(level, r, x, ref)
            assert _noalloc(prob, level, r, x, out) == glls.OK, glls.lib().glls_last_error()
            torch.cuda.synchronize()
            a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
            assert np.abs(a - b).max() <= TOL32 * np.abs(b).max(), (level, call)
            assert np.all(a.reshape(shc)[0] == 0.0)     # coarse boundary rows are zero
    prob.close()


def test_noalloc_rejects_levels_beyond_its_fixed_scratch():
    wl = inputs.terrain2d()                  # fine level: 513 x 513 = 263,169 nodes > 262,144
    prob, _ = glls.problem_for(wl)
    L = prob.levels - 1
    shf, shc = prob.level_shape(L), prob.level_shape(L - 1)
    r = _interior(shf, 1)
    rc = torch.zeros(int(np.prod(shc)), dtype=torch.float32, device="cuda")
    assert _noalloc(prob, L, r, r, rc) == glls.ERR_INVALID
    assert b"262144" in glls.lib().glls_last_error()
    # the next level down fits and works
    sh2, sh1 = prob.level_shape(L - 1), prob.level_shape(L - 2)
    r2 = _interior(sh2, 2)
    out = torch.zeros(int(np.prod(sh1)), dtype=torch.float32, device="cuda")
    ref = torch.zeros_like(out)
    assert _noalloc(prob, L - 1, r2, r2, out) == glls.OK
    prob.restrict(L - 1, r2, r2, ref)
    torch.cuda.synchronize()
    assert (out - ref).abs().max().item() <= TOL32 * ref.abs().max().item()
    prob.close()
