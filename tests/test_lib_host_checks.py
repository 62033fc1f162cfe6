"""tt_ctx_create's host-side argument checks, without a GPU: each case breaks
one rule of include/tt.h on an otherwise valid description and must come back
with its status and message before any CUDA call, leaving the context NULL.
The pointers are placeholders that the checks never dereference."""
import ctypes

import pytest

from paper_2304_11399_gb300 import _lib, build

INV, UNS = _lib.TT_ERR_INVALID_ARG, _lib.TT_ERR_UNSUPPORTED
FAKE = ctypes.c_void_p(0x1000)  # non-NULL placeholder, never read


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _valid():
    g = _lib.Gathers(4, 10, 0, 0, FAKE, FAKE, FAKE)
    p = _lib.ProblemT()
    p.op, p.half_window, p.n_groups, p.n_dom = 1, 5, 1, 2
    p.group_m0 = p.group_dt = p.ap_ptr = p.ap_idx = p.dom_it0 = p.dom_group = FAKE
    c = _lib.DECfg()
    c.np, c.ng, c.F, c.CR, c.seed = 8, 2, 0.5, 0.9, 1
    for k in range(3):
        c.lo[k], c.hi[k] = -1.0, 1.0
    c.exch_every, c.polish_steps, c.polish_lr = 0, 0, 0.0
    return g, p, c


CASES = [
    ("negative size", lambda g, p, c: setattr(g, "ns", -1), INV, b"negative size"),
    ("storage", lambda g, p, c: setattr(g, "storage", 7), INV, b"storage must be"),
    ("operator", lambda g, p, c: setattr(p, "op", 5), INV, b"op must be"),
    ("FO-CRS without h0", lambda g, p, c: setattr(p, "op", 2), INV, b"group_h0"),
    ("half window", lambda g, p, c: setattr(p, "half_window", 9), UNS, b"half_window 9"),
    ("negative half window", lambda g, p, c: setattr(p, "half_window", -1), UNS,
     b"half_window -1"),
    ("NULL traces", lambda g, p, c: setattr(g, "traces", None), INV, b"NULL trace"),
    ("NULL group array", lambda g, p, c: setattr(p, "ap_ptr", None), INV, b"NULL group"),
    ("domains without groups", lambda g, p, c: setattr(p, "n_groups", 0), INV,
     b"no groups"),
    ("negative grid", lambda g, p, c: setattr(p, "n_m0", -1), INV, b"exchange grid"),
    ("oversized record", lambda g, p, c: (setattr(g, "n_traces", 1 << 20),
                                          setattr(g, "ns", 1 << 13)), UNS, b"2^32"),
    ("np too small", lambda g, p, c: setattr(c, "np", 3), INV, b"np 3 outside"),
    ("np too large", lambda g, p, c: setattr(c, "np", 1025), INV, b"np 1025 outside"),
    ("negative ng", lambda g, p, c: setattr(c, "ng", -1), INV, b"ng < 0"),
    ("F out of range", lambda g, p, c: setattr(c, "F", 2.5), INV, b"F must be"),
    ("CR NaN", lambda g, p, c: setattr(c, "CR", float("nan")), INV, b"F must be"),
    ("bounds crossed", lambda g, p, c: c.lo.__setitem__(1, 2.0), INV,
     b"bad bounds in dimension 1"),
    ("infinite bound", lambda g, p, c: c.hi.__setitem__(2, float("inf")), INV,
     b"bad bounds in dimension 2"),
    ("negative exchange", lambda g, p, c: setattr(c, "exch_every", -1), INV,
     b"exchange/polish"),
    ("NaN polish rate", lambda g, p, c: setattr(c, "polish_lr", float("nan")), INV,
     b"exchange/polish"),
    ("adapt flag", lambda g, p, c: setattr(c, "adapt", 2), INV, b"adapt must be"),
    ("adaptive F", lambda g, p, c: (setattr(c, "adapt", 1), setattr(c, "F", 0.0)), INV,
     b"initial F"),
    ("adaptive ng", lambda g, p, c: (setattr(c, "adapt", 1), setattr(c, "ng", (1 << 30) - 1)),
     INV, b"2^30"),
]


@pytest.mark.parametrize("name,breaks,status,msg", CASES, ids=[c[0] for c in CASES])
def test_ctx_create_rejects_on_the_host(lib, name, breaks, status, msg):
    g, p, c = _valid()
    breaks(g, p, c)
    h = ctypes.c_void_p(0x1)
    st = lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(p), ctypes.byref(c),
                           None)
    assert st == status, (name, st, lib.tt_last_error(None))
    assert msg in lib.tt_last_error(None), lib.tt_last_error(None)
    assert not h.value


NULL_CTX_CALLS = [n for n, (res, _) in _lib.SIGNATURES.items()
                  if res is not None and n not in ("tt_last_error", "tt_version",
                                                   "tt_ctx_create", "tt_semblance_eval_noalloc")]


@pytest.mark.parametrize("name", NULL_CTX_CALLS)
def test_every_entry_point_rejects_a_null_context(lib, name):
    """Called with a NULL context (every other argument zero or NULL), each
    entry point returns TT_ERR_INVALID_ARG with a message, touching nothing."""
    _, argtypes = _lib.SIGNATURES[name]
    args = [None if (t is _lib.P or hasattr(t, "contents")) else 0 for t in argtypes]
    st = getattr(lib, name)(*args)
    assert st == INV, (name, st)
    assert lib.tt_last_error(None)


def test_destroy_accepts_null(lib):
    lib.tt_ctx_destroy(None)


NOALLOC_CASES = [
    ("NULL structs", None, INV, b"NULL"),
    ("BF16 storage", lambda g, p: setattr(g, "storage", 1), INV, b"F32"),
    ("FO-CRS", lambda g, p: setattr(p, "op", 2), UNS, b""),
    ("operator", lambda g, p: setattr(p, "op", 9), INV, b"op must be"),
    ("half window", lambda g, p: setattr(p, "half_window", 9), UNS, b"half_window 9"),
    ("negative size", lambda g, p: setattr(p, "n_dom", -1), INV, b"negative size"),
    ("NULL problem array", lambda g, p: setattr(p, "dom_group", None), INV, b"NULL problem"),
    ("NULL traces", lambda g, p: setattr(g, "mid", None), INV, b"NULL trace"),
]


@pytest.mark.parametrize("name,breaks,status,msg", NOALLOC_CASES,
                         ids=[c[0] for c in NOALLOC_CASES])
def test_noalloc_entry_point_rejects_on_the_host(lib, name, breaks, status, msg):
    g, p, _ = _valid()
    if breaks is None:
        st = lib.tt_semblance_eval_noalloc(None, None, FAKE, 1, FAKE, None)
    else:
        breaks(g, p)
        st = lib.tt_semblance_eval_noalloc(ctypes.byref(g), ctypes.byref(p), FAKE, 4, FAKE,
                                           None)
    assert st == status, (name, st, lib.tt_last_error(None))
    assert msg in lib.tt_last_error(None)


def test_noalloc_with_no_domains_is_a_no_op(lib):
    g, p, _ = _valid()
    p.n_dom = 0
    assert lib.tt_semblance_eval_noalloc(ctypes.byref(g), ctypes.byref(p), None, 4, None,
                                         None) == _lib.TT_OK
