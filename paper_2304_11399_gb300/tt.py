"""Python binding of libtt with the same names as the C ABI (include/tt.h).

Argument marshalling only: tensors are checked for device, dtype, shape and
contiguity and passed as raw pointers together with torch's current CUDA
stream; every step of the computation runs in the library's kernels. PyTorch
provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import _lib as L


class TTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t, name, *, dtype=torch.float32, shape=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _check(lib, ctx_handle, status):
    if status != L.TT_OK:
        msg = lib.tt_last_error(ctx_handle).decode()
        raise TTError(status, msg)


def _dev(a, dtype, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


@dataclasses.dataclass
class Context:
    """Owns one tt_ctx (created by :func:`tt_ctx_create`)."""
    handle: C.c_void_p
    n_dom: int
    D: int
    np: int
    n_m0: int
    n_t0: int
    device: torch.device
    lib: C.CDLL

    def close(self):
        if self.handle:
            self.lib.tt_ctx_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tt_version() -> str:
    return L.load().tt_version().decode()


def tt_ctx_create(traces, mid, off, problem, cfg=None, *, storage: str = "f32",
                  device="cuda", stream=None) -> Context:
    """Create a context. ``traces`` [n_tr, ns], ``mid``/``off`` [n_tr] (numpy
    or tensors); ``problem`` has the fields of tt_problem (numpy arrays);
    ``cfg`` has np, ng, F, CR, seed, lo, hi, exch_every, polish_steps,
    polish_lr (or None)."""
    lib = L.load()
    device = torch.device(device)
    tr = _dev(traces, torch.float32, device)
    mid_t = _dev(mid, torch.float32, device)
    off_t = _dev(off, torch.float32, device)
    n_tr, ns = (int(tr.shape[0]), int(tr.shape[1])) if tr.dim() == 2 else (0, 0)
    g = L.Gathers(n_tr, ns, L.TT_STORE_BF16 if storage == "bf16" else L.TT_STORE_F32, 0,
                  tr.data_ptr(), mid_t.data_ptr(), off_t.data_ptr())
    arrs = dict(group_m0=_dev(problem.group_m0, torch.float32, device),
                group_dt=_dev(problem.group_dt, torch.float32, device),
                ap_ptr=_dev(problem.ap_ptr, torch.int32, device),
                ap_idx=_dev(problem.ap_idx, torch.int32, device),
                dom_it0=_dev(problem.dom_it0, torch.int32, device),
                dom_group=_dev(problem.dom_group, torch.int32, device))
    h0 = getattr(problem, "group_h0", None)
    if h0 is not None:
        arrs["group_h0"] = _dev(h0, torch.float32, device)
    n_groups = int(arrs["group_m0"].numel())
    n_dom = int(arrs["dom_it0"].numel())
    p = L.ProblemT(int(problem.op), int(problem.half_window), n_groups, n_dom,
                   *(arrs[k].data_ptr() for k in ("group_m0", "group_dt", "ap_ptr", "ap_idx",
                                                 "dom_it0", "dom_group")),
                   int(getattr(problem, "n_m0", 0)), int(getattr(problem, "n_t0", 0)),
                   arrs["group_h0"].data_ptr() if h0 is not None else None)
    cfg_p = None
    npop = 0
    if cfg is not None:
        c = L.DECfg()
        c.np, c.ng, c.F, c.CR = int(cfg.np), int(cfg.ng), float(cfg.F), float(cfg.CR)
        c.seed = int(cfg.seed) & 0xFFFFFFFFFFFFFFFF
        for k, (lo, hi) in enumerate(zip(cfg.lo, cfg.hi)):
            c.lo[k], c.hi[k] = float(lo), float(hi)
        c.exch_every = int(getattr(cfg, "exch_every", 0))
        c.polish_steps = int(getattr(cfg, "polish_steps", 0))
        c.polish_lr = float(getattr(cfg, "polish_lr", 0.0))
        c.adapt = int(getattr(cfg, "adapt", 0))
        cfg_p = C.byref(c)
        npop = c.np
    h = C.c_void_p()
    with torch.cuda.device(device):
        st = lib.tt_ctx_create(C.byref(h), C.byref(g), C.byref(p), cfg_p, _stream(stream))
    _check(lib, None, st)
    D = {L.TT_OP_CMP: 1, L.TT_OP_CRS: 3, L.TT_OP_FOCRS: 5}[int(problem.op)]
    return Context(h, n_dom, D, npop, int(getattr(problem, "n_m0", 0)),
                   int(getattr(problem, "n_t0", 0)), device, lib)


def tt_ctx_load_traces(ctx: Context, traces, stream=None):
    """Reload the context's traces from a CUDA tensor or a (pinned) CPU tensor."""
    if not isinstance(traces, torch.Tensor) or traces.dtype != torch.float32 \
            or not traces.is_contiguous():
        raise ValueError("traces must be a contiguous float32 tensor")
    host = 0 if traces.is_cuda else 1
    st = ctx.lib.tt_ctx_load_traces(ctx.handle, C.c_void_p(traces.data_ptr()), host,
                                    _stream(stream))
    _check(ctx.lib, ctx.handle, st)


def tt_semblance_eval(ctx: Context, theta: torch.Tensor, S: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """S [n_dom, P] for theta [n_dom, P, D]."""
    if theta.dim() != 3:
        raise ValueError("theta must be [n_dom, P, D]")
    P = int(theta.shape[1])
    tp = _ptr(theta, "theta", shape=(ctx.n_dom, P, ctx.D))
    if S is None:
        S = torch.empty((ctx.n_dom, P), dtype=torch.float32, device=theta.device)
    sp = _ptr(S, "S", shape=(ctx.n_dom, P))
    _check(ctx.lib, ctx.handle, ctx.lib.tt_semblance_eval(ctx.handle, tp, P, sp, _stream(stream)))
    return S


def tt_stack(ctx: Context, theta: torch.Tensor, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """Stacked zero-offset sample out [n_dom] along theta [n_dom, D] (one
    operator per domain, e.g. the best theta of a search)."""
    if theta.dim() == 3 and theta.shape[1] == 1:
        theta = theta[:, 0]
    tp = _ptr(theta, "theta", shape=(ctx.n_dom, ctx.D))
    if out is None:
        out = torch.empty((ctx.n_dom,), dtype=torch.float32, device=theta.device)
    op = _ptr(out, "out", shape=(ctx.n_dom,))
    _check(ctx.lib, ctx.handle, ctx.lib.tt_stack(ctx.handle, tp, op, _stream(stream)))
    return out


def tt_semblance_grad(ctx: Context, theta: torch.Tensor, stream=None):
    """(S [n_dom, P], dS/dtheta [n_dom, P, D]) for theta [n_dom, P, D]."""
    P = int(theta.shape[1])
    tp = _ptr(theta, "theta", shape=(ctx.n_dom, P, ctx.D))
    S = torch.empty((ctx.n_dom, P), dtype=torch.float32, device=theta.device)
    dS = torch.empty((ctx.n_dom, P, ctx.D), dtype=torch.float32, device=theta.device)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_semblance_grad(
        ctx.handle, tp, P, C.c_void_p(S.data_ptr()), C.c_void_p(dS.data_ptr()), _stream(stream)))
    return S, dS


def tt_de_step(ctx: Context, gen: int, pop, fit=None, trial=None, trial_fit=None,
               next_trial=None, best_idx=None, stream=None):
    """One DE step in place (see include/tt.h); returns (pop, fit, next_trial, best_idx)."""
    shp = (ctx.n_dom, ctx.np, ctx.D)
    pp = _ptr(pop, "pop", shape=shp)
    fp = _ptr(fit, "fit", shape=shp[:2], allow_none=gen == 0)
    tp = _ptr(trial, "trial", shape=shp, allow_none=True)
    tfp = _ptr(trial_fit, "trial_fit", shape=shp[:2], allow_none=True)
    np_ = _ptr(next_trial, "next_trial", shape=shp, allow_none=True)
    bp = _ptr(best_idx, "best_idx", dtype=torch.int32, shape=(ctx.n_dom,), allow_none=True)
    _check(ctx.lib, ctx.handle,
           ctx.lib.tt_de_step(ctx.handle, int(gen), pp, fp, tp, tfp, np_, bp, _stream(stream)))
    return pop, fit, next_trial, best_idx


def tt_jade_state(ctx: Context, state: dict | None = None, stream=None) -> dict:
    """Save (state None: returns new tensors mu, n_arc, archive, F, CR) or
    restore (state given) the context's JADE adaptation state."""
    n, NP, D = ctx.n_dom, ctx.np, ctx.D
    shapes = dict(mu=((n, 2), torch.float32), n_arc=((n,), torch.int32),
                  archive=((n, NP, D), torch.float32), F=((n, NP), torch.float32),
                  CR=((n, NP), torch.float32))
    save = state is None
    if save:
        state = {k: torch.empty(s, dtype=dt, device=ctx.device) for k, (s, dt) in shapes.items()}
    ptrs = [_ptr(state[k], k, dtype=dt, shape=s) for k, (s, dt) in shapes.items()]
    _check(ctx.lib, ctx.handle,
           ctx.lib.tt_jade_state(ctx.handle, 1 if save else 0, *ptrs, _stream(stream)))
    return state


def tt_best_snapshot(ctx: Context, pop, fit, stream=None):
    """(best_theta [n_dom, D], best_S [n_dom]) of a population."""
    bt = torch.empty((ctx.n_dom, ctx.D), dtype=torch.float32, device=pop.device)
    bs = torch.empty((ctx.n_dom,), dtype=torch.float32, device=pop.device)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_best_snapshot(
        ctx.handle, _ptr(pop, "pop", shape=(ctx.n_dom, ctx.np, ctx.D)),
        _ptr(fit, "fit", shape=(ctx.n_dom, ctx.np)), C.c_void_p(bt.data_ptr()),
        C.c_void_p(bs.data_ptr()), _stream(stream)))
    return bt, bs


def tt_neighbor_exchange(ctx: Context, n_m0: int, n_t0: int, best_theta, pop, fit, stream=None):
    """In-place exchange; returns (imports [n_dom, 4, D], slots [n_dom, 4])."""
    imports = torch.empty((ctx.n_dom, 4, ctx.D), dtype=torch.float32, device=pop.device)
    slots = torch.empty((ctx.n_dom, 4), dtype=torch.int32, device=pop.device)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_neighbor_exchange(
        ctx.handle, int(n_m0), int(n_t0), _ptr(best_theta, "best_theta", shape=(ctx.n_dom, ctx.D)),
        _ptr(pop, "pop", shape=(ctx.n_dom, ctx.np, ctx.D)),
        _ptr(fit, "fit", shape=(ctx.n_dom, ctx.np)), C.c_void_p(imports.data_ptr()),
        C.c_void_p(slots.data_ptr()), _stream(stream)))
    return imports, slots


def tt_polish(ctx: Context, theta, steps: int, lr: float, stream=None):
    """Polish theta [n_dom, D] in place; returns (theta, S)."""
    S = torch.empty((ctx.n_dom,), dtype=torch.float32, device=theta.device)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_polish(
        ctx.handle, _ptr(theta, "theta", shape=(ctx.n_dom, ctx.D)), C.c_void_p(S.data_ptr()),
        int(steps), float(lr), _stream(stream)))
    return theta, S


def tt_search(ctx: Context, best_theta=None, best_S=None, stream=None):
    """Whole search; returns (best_theta [n_dom, D], best_S [n_dom], n_evals)."""
    if best_theta is None:
        best_theta = torch.empty((ctx.n_dom, ctx.D), dtype=torch.float32, device=ctx.device)
    if best_S is None:
        best_S = torch.empty((ctx.n_dom,), dtype=torch.float32, device=ctx.device)
    n = C.c_uint64(0)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_search(
        ctx.handle, _ptr(best_theta, "best_theta", shape=(ctx.n_dom, ctx.D)),
        _ptr(best_S, "best_S", shape=(ctx.n_dom,)), C.byref(n), _stream(stream)))
    return best_theta, best_S, int(n.value)


def tt_search_slab(ctx: Context, dom_base: int, has_prev: bool, has_next: bool, exchange=None,
                   best_theta=None, best_S=None, stream=None):
    """The search on one slab of a sharded line (see include/tt.h, tt_slab).
    ``exchange(gen, send_first, send_last, recv_prev, recv_next)`` receives
    four [n_t0, D] device tensors: it sends the first two to the previous and
    next slab and fills the last two with theirs (e.g.
    ``slab.halo_exchange``). Returns (best_theta, best_S, n_evals)."""
    if best_theta is None:
        best_theta = torch.empty((ctx.n_dom, ctx.D), dtype=torch.float32, device=ctx.device)
    if best_S is None:
        best_S = torch.empty((ctx.n_dom,), dtype=torch.float32, device=ctx.device)
    rows = [torch.zeros((ctx.n_t0, ctx.D), dtype=torch.float32, device=ctx.device)
            for _ in range(4)]
    failure = []

    def trampoline(user, gen, stream_ptr):
        try:
            exchange(int(gen), *rows)
            return 0
        except BaseException as e:  # re-raised below, after the library returns
            failure.append(e)
            return 1

    fn = L.HaloFn(trampoline) if exchange is not None else L.HaloFn()
    sl = L.Slab(int(dom_base), 1 if has_prev else 0, 1 if has_next else 0,
                *(C.c_void_p(t.data_ptr()) for t in rows), fn, None)
    n = C.c_uint64(0)
    st = ctx.lib.tt_search_slab(ctx.handle, C.byref(sl),
                                _ptr(best_theta, "best_theta", shape=(ctx.n_dom, ctx.D)),
                                _ptr(best_S, "best_S", shape=(ctx.n_dom,)), C.byref(n),
                                _stream(stream))
    if failure:
        raise failure[0]
    _check(ctx.lib, ctx.handle, st)
    return best_theta, best_S, int(n.value)


def tt_ens_search(ctx: Context, np_f: int = 5, ng_f: int = 1, np_bf: int = 5, ng_bf: int = 1,
                  n_skip: int = 2, n_cycle: int = 1, n_bucket: int = 64, best_theta=None,
                  best_S=None, stream=None):
    """ENS sweep mode; returns (best_theta [n_dom, D], best_S [n_dom], n_evals)."""
    e = L.EnsCfg(int(np_f), int(ng_f), int(np_bf), int(ng_bf), int(n_skip), int(n_cycle),
                 int(n_bucket), 0)
    if best_theta is None:
        best_theta = torch.empty((ctx.n_dom, ctx.D), dtype=torch.float32, device=ctx.device)
    if best_S is None:
        best_S = torch.empty((ctx.n_dom,), dtype=torch.float32, device=ctx.device)
    n = C.c_uint64(0)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ens_search(
        ctx.handle, C.byref(e), _ptr(best_theta, "best_theta", shape=(ctx.n_dom, ctx.D)),
        _ptr(best_S, "best_S", shape=(ctx.n_dom,)), C.byref(n), _stream(stream)))
    return best_theta, best_S, int(n.value)


_KERNELS = {"packed": L.TT_KERNEL_PACKED, "persistent": L.TT_KERNEL_PERSISTENT,
            "scalar": L.TT_KERNEL_SCALAR}


def tt_ctx_set_option(ctx: Context, option: str, value):
    """option: "kernel" ("packed" | "persistent" | "scalar"), "block" (128 | 256),
    "search_graph" (bool), "split" (bool: split the aperture over the warps
    of a block for launches of fewer than the "split_max_pairs" threshold) or
    "member_order" (True: the search evaluates each domain's members in the
    order of their window position, same results; False: index order;
    "auto", the default: True when the apertures hold at least 768 traces
    on average)."""
    if option == "kernel":
        code, v = L.TT_OPT_KERNEL, _KERNELS[value]
    elif option == "block":
        code, v = L.TT_OPT_BLOCK, int(value)
    elif option == "search_graph":
        code, v = L.TT_OPT_SEARCH_GRAPH, 1 if value else 0
    elif option == "split":
        code, v = L.TT_OPT_SPLIT, 1 if value else 0
    elif option == "member_order":
        code, v = L.TT_OPT_MEMBER_ORDER, 2 if value == "auto" else (1 if value else 0)
    else:
        raise ValueError(f"unknown option {option}")
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_set_option(ctx.handle, code, v))


def tt_ctx_get_option(ctx: Context, option: str):
    """option: as for tt_ctx_set_option, or the read-only "split_max_pairs"
    (split threshold in pairs) and "sm_count" (the device's multiprocessors)."""
    code = {"kernel": L.TT_OPT_KERNEL, "block": L.TT_OPT_BLOCK,
            "search_graph": L.TT_OPT_SEARCH_GRAPH, "split": L.TT_OPT_SPLIT,
            "member_order": L.TT_OPT_MEMBER_ORDER,
            "split_max_pairs": L.TT_OPT_SPLIT_MAX_PAIRS, "sm_count": L.TT_OPT_SM_COUNT}[option]
    v = C.c_int64()
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_get_option(ctx.handle, code, C.byref(v)))
    if option == "kernel":
        return {b: a for a, b in _KERNELS.items()}[v.value]
    if option == "member_order":
        return "auto" if v.value == 2 else bool(v.value)
    return bool(v.value) if option in ("search_graph", "split") else int(v.value)


def tt_ctx_autotune(ctx: Context, theta: torch.Tensor, stream=None):
    """Time every kernel variant on theta [n_dom, P, D] and keep the fastest,
    except that a persistent variant is kept only when it is more than 3%
    faster than the fastest packed or scalar one. Returns {(variant, block): ms}."""
    P = int(theta.shape[1])
    tp = _ptr(theta, "theta", shape=(ctx.n_dom, P, ctx.D))
    S = torch.empty((ctx.n_dom, P), dtype=torch.float32, device=theta.device)
    times = (C.c_float * L.TT_N_TUNE_CANDIDATES)()
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_autotune(ctx.handle, tp, P, C.c_void_p(S.data_ptr()),
                                                        times, _stream(stream)))
    return {cand: float(times[i]) for i, cand in enumerate(L.TUNE_CANDIDATES)}


def tt_ctx_profile(ctx: Context, enable: bool = True):
    """Enable or disable event timing of the context's semblance launches."""
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_profile(ctx.handle, 1 if enable else 0))


def tt_ctx_probe_l1(ctx: Context, iters: int = 4000, stream=None) -> float:
    """Enqueue the L1 load-bandwidth probe; returns the bytes it loads (time
    it with CUDA events on the stream)."""
    b = C.c_double(0.0)
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_probe_l1(ctx.handle, int(iters), C.byref(b),
                                                        _stream(stream)))
    return b.value


def tt_ctx_stats(ctx: Context, reset: bool = False) -> dict:
    """Launch counters and the summed device time of semblance launches."""
    st = L.Stats()
    _check(ctx.lib, ctx.handle, ctx.lib.tt_ctx_stats(ctx.handle, C.byref(st), 1 if reset else 0))
    return {k: getattr(st, k) for k, _ in L.Stats._fields_}


class SemblanceFn(torch.autograd.Function):
    """S(theta) with the hand-written adjoint kernel as its backward."""

    @staticmethod
    def forward(fctx, ctx: Context, theta: torch.Tensor):
        theta = theta.contiguous()
        fctx.tt = ctx
        fctx.save_for_backward(theta)
        return tt_semblance_eval(ctx, theta)

    @staticmethod
    def backward(fctx, gS):
        (theta,) = fctx.saved_tensors
        _, dS = tt_semblance_grad(fctx.tt, theta)
        return None, gS.unsqueeze(-1) * dS


def semblance(ctx: Context, theta: torch.Tensor) -> torch.Tensor:
    """Differentiable S [n_dom, P] of theta [n_dom, P, D]."""
    return SemblanceFn.apply(ctx, theta)
