"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/glls.h (no device work is done here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_10710_gb300 import glls
    return glls.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "glls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glls_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_library_gll_matches_oracle(lib):
    from oracle import gll as ogll
    from paper_2504_10710_gb300 import glls
    for p in (1, 2, 3, 7, 8, 12, 24):
        xi, rho = glls.gll(p)
        xo, ro = ogll.gll(p)
        np.testing.assert_allclose(xi, xo, atol=2e-16)
        np.testing.assert_allclose(rho, ro, atol=2e-16)


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_2504_10710_gb300 import glls
    with pytest.raises(glls.GllsError) as ei:
        glls.gll(0)
    assert ei.value.status == glls.ERR_INVALID
    with pytest.raises(glls.GllsError) as ei:
        glls.Problem(4, (2, 2), 3, np.zeros((4, 49)))
    assert ei.value.status == glls.ERR_INVALID
    assert lib.glls_last_error() != b""


def test_no_device_gives_an_error_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2504_10710_gb300 import glls, inputs
    wl = inputs.random2d((2, 2), 3)
    xi, _ = glls.gll(3)
    with pytest.raises(glls.GllsError) as ei:
        glls.Problem(2, (2, 2), 3, wl.coords(xi))
    assert ei.value.status == glls.ERR_CUDA
