"""libtt builds, loads without a GPU and exports every function tt.h declares."""
import ctypes
import os

import pytest

from paper_2304_11399_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _lib.header_declarations(os.path.join(ROOT, "include", "tt.h"))
    for required in ("tt_semblance_eval", "tt_semblance_grad", "tt_de_step",
                     "tt_neighbor_exchange", "tt_search"):
        assert required in names
    assert len(set(names)) == len(names)


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_declarations(os.path.join(ROOT, "include", "tt.h"))
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_version_and_error_without_gpu(lib):
    assert b"sm_103a" in lib.tt_version()
    # invalid arguments are rejected on the host before any CUDA call
    h = ctypes.c_void_p()
    st = lib.tt_ctx_create(ctypes.byref(h), None, None, None, None)
    assert st == _lib.TT_ERR_INVALID_ARG
    assert b"NULL" in lib.tt_last_error(None)
    assert lib.tt_semblance_eval(None, None, 1, None, None) == _lib.TT_ERR_INVALID_ARG
    assert lib.tt_search(None, None, None, None, None) == _lib.TT_ERR_INVALID_ARG
    g = _lib.Gathers(4, 10, 7, 0, None, None, None)
    p = _lib.ProblemT()
    assert lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(p), None,
                             None) == _lib.TT_ERR_INVALID_ARG
    g.storage = 0
    p.op = 1
    p.half_window = 9
    assert lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(p), None,
                             None) == _lib.TT_ERR_UNSUPPORTED
    assert not h.value


def test_binding_struct_layout_matches_header(tmp_path):
    """The ctypes structs against the C compiler's layout of include/tt.h:
    size and every field offset."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"tt_gathers": _lib.Gathers, "tt_problem": _lib.ProblemT,
               "tt_de_cfg": _lib.DECfg, "tt_ens_cfg": _lib.EnsCfg, "tt_stats": _lib.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tt.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, *_ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            *key, val = ln.split()
            got[tuple(key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, *_ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_package_has_no_cpu_fallback():
    import paper_2304_11399_gb300.tt as t
    src = open(t.__file__).read()
    assert "oracle" not in src and "numpy.linalg" not in src
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(os.path.join(ROOT, "does_not_exist", "libtt.so"))
