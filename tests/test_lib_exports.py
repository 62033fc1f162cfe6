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


def test_binding_struct_layout_matches_header():
    # natural C alignment of the three structs, as laid out in tt.h
    assert ctypes.sizeof(_lib.Gathers) == 40
    assert ctypes.sizeof(_lib.ProblemT) == 72
    assert _lib.DECfg.seed.offset == 16
    assert _lib.DECfg.exch_every.offset == 88
    assert ctypes.sizeof(_lib.DECfg) == 104


def test_package_has_no_cpu_fallback():
    import paper_2304_11399_gb300.tt as t
    src = open(t.__file__).read()
    assert "oracle" not in src and "numpy.linalg" not in src
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(os.path.join(ROOT, "does_not_exist", "libtt.so"))
