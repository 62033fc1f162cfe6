"""The allocation-free entry point, tt_semblance_eval_noalloc, through the C ABI.

It serves callers that cannot allocate device memory (their host
application owns every device buffer, or cudaMalloc is not allowed once
their service loop runs) and therefore cannot create a context. It must
give what tt_semblance_eval gives on the same inputs, within the FP32
parity tolerance of the other tests (|dS| <= 1e-5), also when two calls
follow each other and share the library's fixed scratch array. This file is
collected last so that a run stopping at its first failure has run
everything else first; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2304_11399_gb300 as tt
from paper_2304_11399_gb300 import _lib
from gpu_util import dev, random_theta, to_dev, small_line, configs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _cabi_args(traces, mid, off, prob):
    """Device copies of the inputs and the tt_gathers / tt_problem structs."""
    keep = dict(traces=to_dev(traces), mid=to_dev(mid), off=to_dev(off),
                group_m0=to_dev(prob.group_m0), group_dt=to_dev(prob.group_dt),
                ap_ptr=to_dev(prob.ap_ptr, torch.int32), ap_idx=to_dev(prob.ap_idx, torch.int32),
                dom_it0=to_dev(prob.dom_it0, torch.int32),
                dom_group=to_dev(prob.dom_group, torch.int32))
    g = _lib.Gathers(int(traces.shape[0]), int(traces.shape[1]), _lib.TT_STORE_F32, 0,
                     keep["traces"].data_ptr(), keep["mid"].data_ptr(), keep["off"].data_ptr())
    p = _lib.ProblemT(int(prob.op), int(prob.half_window), int(prob.group_m0.size),
                      int(prob.dom_it0.size),
                      *(keep[k].data_ptr() for k in ("group_m0", "group_dt", "ap_ptr", "ap_idx",
                                                    "dom_it0", "dom_group")), 0, 0)
    return g, p, keep


def _noalloc(lib, g, p, theta_t, S_t):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.tt_semblance_eval_noalloc(C.byref(g), C.byref(p), C.c_void_p(theta_t.data_ptr()),
                                         int(theta_t.shape[1]), C.c_void_p(S_t.data_ptr()),
                                         stream)


def _context_eval(traces, mid, off, prob, theta):
    ctx = tt.tt_ctx_create(traces, mid, off, prob, None, device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    return S


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    lib = _lib.load()
    # call 1: a CRS line (uneven apertures clipped at the line ends, P = 20)
    wa = small_line(21)
    ta = random_theta(wa.problem.n_dom, 20, wa.de.lo, wa.de.hi, 1)
    # call 2: the CMP gather, every sample, P = 7 (rewrites the shared scratch)
    wb = configs.cmp_search(2)
    tb = random_theta(wb.problem.n_dom, 7, wb.de.lo, wb.de.hi, 2)
    ga, pa, ka = _cabi_args(wa.traces, wa.mid, wa.off, wa.problem)
    gb, pb, kb = _cabi_args(wb.traces, wb.mid, wb.off, wb.problem)
    ta_t, tb_t = to_dev(ta), to_dev(tb)
    Sa = torch.full((wa.problem.n_dom, 20), -1.0, device=dev())
    Sb = torch.full((wb.problem.n_dom, 7), -1.0, device=dev())
    assert _noalloc(lib, ga, pa, ta_t, Sa) == _lib.TT_OK, lib.tt_last_error(None)
    assert _noalloc(lib, gb, pb, tb_t, Sb) == _lib.TT_OK, lib.tt_last_error(None)
    torch.cuda.synchronize()
    ref_a = _context_eval(wa.traces, wa.mid, wa.off, wa.problem, ta)
    ref_b = _context_eval(wb.traces, wb.mid, wb.off, wb.problem, tb)
    assert np.max(np.abs(Sa.cpu().numpy() - ref_a)) <= TOL
    assert np.max(np.abs(Sb.cpu().numpy() - ref_b)) <= TOL
    # the same call again after the other one: same answer as the first time
    Sa2 = torch.full_like(Sa, -1.0)
    assert _noalloc(lib, ga, pa, ta_t, Sa2) == _lib.TT_OK
    torch.cuda.synchronize()
    assert torch.equal(Sa, Sa2)


def test_noalloc_rejects_oversize_and_invalid_input():
    lib = _lib.load()
    wl = small_line(22, n_cmp=3, ns=60, ap_half=1)
    prob = wl.problem
    # an aperture list one entry longer than the fixed scratch holds
    n_big = _lib.TT_NOALLOC_MAX_APERTURE_ENTRIES + 1
    big = synth.Problem(op=1, half_window=5, group_m0=np.zeros(1, np.float32),
                        group_dt=np.full(1, 0.004, np.float32),
                        ap_ptr=np.array([0, n_big], np.int32), ap_idx=np.zeros(n_big, np.int32),
                        dom_it0=np.zeros(1, np.int32), dom_group=np.zeros(1, np.int32))
    g, p, keep = _cabi_args(wl.traces, wl.mid, wl.off, big)
    th = torch.zeros((1, 1, 3), device=dev())
    S = torch.zeros((1, 1), device=dev())
    assert _noalloc(lib, g, p, th, S) == _lib.TT_ERR_UNSUPPORTED
    assert b"at most" in lib.tt_last_error(None)
    # the FO-CRS operator is evaluated through a context only
    fo = synth.Problem(**{**prob.__dict__})
    fo.op = _lib.TT_OP_FOCRS
    g, p, keep = _cabi_args(wl.traces, wl.mid, wl.off, fo)
    assert _noalloc(lib, g, p, th, S) == _lib.TT_ERR_UNSUPPORTED
    assert b"TT_OP_CRS only" in lib.tt_last_error(None)
    # an out-of-range trace index is caught on the device and reported
    bad = synth.Problem(**{**prob.__dict__})
    bad.ap_idx = prob.ap_idx.copy()
    bad.ap_idx[5] = wl.traces.shape[0]
    g, p, keep = _cabi_args(wl.traces, wl.mid, wl.off, bad)
    th = to_dev(random_theta(prob.n_dom, 2, wl.de.lo, wl.de.hi, 3))
    S = torch.zeros((prob.n_dom, 2), device=dev())
    assert _noalloc(lib, g, p, th, S) == _lib.TT_ERR_INVALID_ARG
    assert b"ap_idx" in lib.tt_last_error(None)


def test_noalloc_long_record_matches_oracle():
    """3000-sample records at 2 ms: window centres near u = 3000 samples,
    where FP32 rounding of u itself would move S by ~2e-5. The entry point
    takes the moveout form of the position there and stays within 1e-5 of
    the FP64 oracle, and of the context path, on two calls in a row."""
    import oracle
    lib = _lib.load()
    wl = configs.large_line(31, n_cmp=5, ns=3000, n_events=12, ap_half=2, cmps=[2],
                            t0_range=(2300, 3000))
    prob = wl.problem
    rng = np.random.default_rng(4)
    theta = random_theta(prob.n_dom, 4, wl.de.lo, wl.de.hi, 5)
    # and the generating parameters of the events, recentred to the CMP, at
    # their own zero-offset samples (semblance near 1 there)
    for ev in wl.line.events:
        t = synth.crs_recentre(ev, wl.line.cmp_x[2])
        if t is None:
            continue
        it = int(round(t[0] / wl.dt))
        if 2300 <= it < 3000:
            theta[it - 2300, rng.integers(4)] = t[1:4]
    g, p, keep = _cabi_args(wl.traces, wl.mid, wl.off, prob)
    th = to_dev(theta)
    S1 = torch.full((prob.n_dom, 4), -1.0, device=dev())
    S2 = torch.full((prob.n_dom, 4), -1.0, device=dev())
    assert _noalloc(lib, g, p, th, S1) == _lib.TT_OK, lib.tt_last_error(None)
    assert _noalloc(lib, g, p, th, S2) == _lib.TT_OK, lib.tt_last_error(None)
    torch.cuda.synchronize()
    S1, S2 = S1.cpu().numpy(), S2.cpu().numpy()
    assert np.array_equal(S1, S2)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert ref.max() > 0.2  # the events are found: not only noise is compared
    assert np.max(np.abs(S1 - ref)) <= TOL
    assert np.max(np.abs(S1 - _context_eval(wl.traces, wl.mid, wl.off, prob, theta))) <= TOL


@pytest.mark.parametrize("case,needle", [
    ("ap_ptr", b"non-decreasing"), ("dt", b"dt"), ("dom_group", b"dom_group"),
    ("dom_it0", b"dom_it0")])
def test_noalloc_device_validation_flags(case, needle):
    """Each input error that only the device-side validation sees is
    reported as TT_ERR_INVALID_ARG with its own message, before the table
    is built or any sample is read: a decreasing ap_ptr (the check that
    keeps the table's writes inside the fixed scratch array), a zero dt, a
    domain's group equal to n_groups and an it0 of 2^24."""
    lib = _lib.load()
    wl = small_line(23, n_cmp=4, ns=80, ap_half=1)
    bad = synth.Problem(**{**wl.problem.__dict__})
    if case == "ap_ptr":
        bad.ap_ptr = wl.problem.ap_ptr.copy()
        bad.ap_ptr[1] = bad.ap_ptr[2] + 1  # ends still 0 and nnz
    elif case == "dt":
        bad.group_dt = wl.problem.group_dt.copy()
        bad.group_dt[1] = 0.0
    elif case == "dom_group":
        bad.dom_group = wl.problem.dom_group.copy()
        bad.dom_group[7] = bad.group_m0.size
    else:
        bad.dom_it0 = wl.problem.dom_it0.copy()
        bad.dom_it0[3] = 1 << 24
    g, p, keep = _cabi_args(wl.traces, wl.mid, wl.off, bad)
    th = to_dev(random_theta(bad.n_dom, 2, wl.de.lo, wl.de.hi, 6))
    S = torch.full((bad.n_dom, 2), -1.0, device=dev())
    assert _noalloc(lib, g, p, th, S) == _lib.TT_ERR_INVALID_ARG
    assert needle in lib.tt_last_error(None)
    torch.cuda.synchronize()
    assert torch.all(S == -1.0)  # nothing written
