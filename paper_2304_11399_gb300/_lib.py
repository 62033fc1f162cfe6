"""ctypes view of the C ABI declared in include/tt.h (no logic here)."""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtt.so")

TT_OK, TT_ERR_INVALID_ARG, TT_ERR_CUDA, TT_ERR_OUT_OF_MEMORY, TT_ERR_TIMEOUT, \
    TT_ERR_UNSUPPORTED = range(6)
TT_OP_CMP, TT_OP_CRS, TT_OP_FOCRS = 0, 1, 2
TT_OPT_KERNEL, TT_OPT_BLOCK, TT_OPT_SEARCH_GRAPH, TT_OPT_SPLIT = 1, 2, 3, 4
TT_OPT_SPLIT_MAX_PAIRS, TT_OPT_SM_COUNT, TT_OPT_MEMBER_ORDER = 5, 6, 7
TT_KERNEL_PACKED, TT_KERNEL_PERSISTENT, TT_KERNEL_SCALAR = 1, 2, 3
TT_N_TUNE_CANDIDATES = 6
TUNE_CANDIDATES = [("packed", 256), ("packed", 128), ("persistent", 256), ("persistent", 128),
                   ("scalar", 256), ("scalar", 128)]
TT_STORE_F32, TT_STORE_BF16 = 0, 1
TT_MAX_DIM = 8
TT_NOALLOC_SCRATCH_BYTES = 4 << 20
TT_NOALLOC_MAX_APERTURE_ENTRIES = 262128

STATUS_NAMES = {0: "TT_OK", 1: "TT_ERR_INVALID_ARG", 2: "TT_ERR_CUDA",
                3: "TT_ERR_OUT_OF_MEMORY", 4: "TT_ERR_TIMEOUT", 5: "TT_ERR_UNSUPPORTED"}

# every function the header declares: name -> (restype, argtypes)
P = C.c_void_p
I32 = C.c_int32


class Gathers(C.Structure):
    _fields_ = [("n_traces", I32), ("ns", I32), ("storage", I32), ("reserved", I32),
                ("traces", P), ("mid", P), ("off", P)]


class ProblemT(C.Structure):
    _fields_ = [("op", I32), ("half_window", I32), ("n_groups", I32), ("n_dom", I32),
                ("group_m0", P), ("group_dt", P), ("ap_ptr", P), ("ap_idx", P),
                ("dom_it0", P), ("dom_group", P), ("n_m0", I32), ("n_t0", I32),
                ("group_h0", P)]


class DECfg(C.Structure):
    _fields_ = [("np", I32), ("ng", I32), ("F", C.c_float), ("CR", C.c_float),
                ("seed", C.c_uint64), ("lo", C.c_float * TT_MAX_DIM),
                ("hi", C.c_float * TT_MAX_DIM), ("exch_every", I32), ("polish_steps", I32),
                ("polish_lr", C.c_float), ("adapt", I32)]


class EnsCfg(C.Structure):
    _fields_ = [("np_f", I32), ("ng_f", I32), ("np_bf", I32), ("ng_bf", I32), ("n_skip", I32),
                ("n_cycle", I32), ("n_bucket", I32), ("reserved", I32)]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("semblance_launches", C.c_uint64),
                ("trace_evals", C.c_double), ("semblance_ms", C.c_double),
                ("timed_launches", C.c_uint64)]


HaloFn = C.CFUNCTYPE(I32, P, I32, P)


class Slab(C.Structure):
    _fields_ = [("dom_base", C.c_int64), ("has_prev", I32), ("has_next", I32),
                ("send_first", P), ("send_last", P), ("recv_prev", P), ("recv_next", P),
                ("exchange", HaloFn), ("user", P)]


SIGNATURES = {
    "tt_last_error": (C.c_char_p, [P]),
    "tt_version": (C.c_char_p, []),
    "tt_ctx_create": (I32, [C.POINTER(P), C.POINTER(Gathers), C.POINTER(ProblemT),
                            C.POINTER(DECfg), P]),
    "tt_ctx_load_traces": (I32, [P, P, I32, P]),
    "tt_ctx_destroy": (None, [P]),
    "tt_semblance_eval": (I32, [P, P, I32, P, P]),
    "tt_semblance_grad": (I32, [P, P, I32, P, P, P]),
    "tt_stack": (I32, [P, P, P, P]),
    "tt_jade_state": (I32, [P, I32, P, P, P, P, P, P]),
    "tt_de_step": (I32, [P, I32, P, P, P, P, P, P, P]),
    "tt_best_snapshot": (I32, [P, P, P, P, P, P]),
    "tt_neighbor_exchange": (I32, [P, I32, I32, P, P, P, P, P, P]),
    "tt_polish": (I32, [P, P, P, I32, C.c_float, P]),
    "tt_search": (I32, [P, P, P, C.POINTER(C.c_uint64), P]),
    "tt_search_slab": (I32, [P, C.POINTER(Slab), P, P, C.POINTER(C.c_uint64), P]),
    "tt_ctx_profile": (I32, [P, I32]),
    "tt_ctx_stats": (I32, [P, C.POINTER(Stats), I32]),
    "tt_ctx_probe_l1": (I32, [P, I32, C.POINTER(C.c_double), P]),
    "tt_semblance_eval_noalloc": (I32, [C.POINTER(Gathers), C.POINTER(ProblemT), P, I32, P, P]),
    "tt_ctx_set_option": (I32, [P, I32, C.c_int64]),
    "tt_ctx_get_option": (I32, [P, I32, C.POINTER(C.c_int64)]),
    "tt_ctx_autotune": (I32, [P, P, I32, P, C.POINTER(C.c_float), P]),
    "tt_ens_search": (I32, [P, C.POINTER(EnsCfg), P, P, C.POINTER(C.c_uint64), P]),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libtt.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libtt.so is not built ({p}); run __graft_entry__.build() — "
                           "there is no CPU fallback")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def header_declarations(header_path: str) -> list[str]:
    """Names of the functions declared in a C header (for export checks)."""
    import re
    txt = open(header_path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tt_[a-z_0-9]+)\s*\(", txt, flags=re.M)
