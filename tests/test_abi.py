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


# (C struct, ctypes class) pairs of the binding; every field's offset and the
# struct size must agree with what a C compiler makes of include/glls.h
STRUCTS = [("glls_mesh_desc", "MeshDesc"), ("glls_solve_opts", "SolveOpts"), ("glls_stats", "Stats"),
           ("glls_info", "Info"), ("glls_server_info", "ServerInfo")]


def _c_layout(tmp_path):
    """Compile a C probe against the header: sizeof and offsetof of every
    field the binding declares."""
    import shutil
    import subprocess
    from paper_2504_10710_gb300 import glls
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include "glls.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, pyname in STRUCTS:
        lines.append(f'    printf("{pyname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(glls, pyname)._fields_:
            lines.append(f'    printf("{pyname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_binding_struct_layouts_match_the_header(tmp_path):
    from paper_2504_10710_gb300 import glls
    c = _c_layout(tmp_path)
    for _, pyname in STRUCTS:
        cls = getattr(glls, pyname)
        assert c[(pyname, "size")] == ctypes.sizeof(cls), pyname
        for fname, _ in cls._fields_:
            assert c[(pyname, fname)] == getattr(cls, fname).offset, (pyname, fname)


def test_binding_constants_match_the_header():
    """Every enum constant of include/glls.h has the value the binding uses."""
    from paper_2504_10710_gb300 import glls
    src = open(os.path.join(ROOT, "include", "glls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\bGLLS_(\w+)\s*=\s*(-?\d+)", src)}
    assert len(consts) >= 20
    for name, value in consts.items():
        assert hasattr(glls, name), name
        assert getattr(glls, name) == value, (name, getattr(glls, name), value)


def test_bad_summation_rejected_before_device_work(lib):
    from paper_2504_10710_gb300 import glls, inputs
    wl = inputs.random2d((2, 2), 3)
    xi, _ = glls.gll(3)
    with pytest.raises(glls.GllsError) as ei:
        glls.Problem(2, (2, 2), 3, wl.coords(xi), summation=5)
    assert ei.value.status == glls.ERR_INVALID
    assert b"summation" in lib.glls_last_error()
