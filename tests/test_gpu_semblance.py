"""GPU semblance (tt_semblance_eval) against the FP64 oracle, through the C ABI.

Tolerance: |dS| <= 1e-5 for FP32-stored traces (the stated bound for the
FP32 path); BF16-stored traces are compared with the oracle on the same
BF16-rounded record at 1e-5 and with the FP32 record at 2e-3.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, random_theta, to_dev, bf16_round, small_line, synth, configs

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _eval(wl_traces, mid, off, prob, theta, storage="f32"):
    ctx = tt.tt_ctx_create(wl_traces, mid, off, prob, None, storage=storage, device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    return S


def test_hand_worked_cases_through_cabi(golden_dir):
    from test_oracle_semblance import load_worked
    for c in load_worked(os.path.join(golden_dir, "semblance_worked.txt")):
        m = np.array([t[0] for t in c["traces"]], np.float32)
        h = np.array([t[1] for t in c["traces"]], np.float32)
        ns = max(len(t) - 2 for t in c["traces"])
        x = np.zeros((len(m), ns), np.float32)
        for i, t in enumerate(c["traces"]):
            x[i, :len(t) - 2] = t[2:]
        prob = synth.Problem(op=c["op"], half_window=c["w"],
                             group_m0=np.array([c["m0"]], np.float32),
                             group_dt=np.array([c["dt"]], np.float32),
                             ap_ptr=np.array([0, len(m)], np.int32),
                             ap_idx=np.arange(len(m), dtype=np.int32),
                             dom_it0=np.array([c["it0"]], np.int32),
                             dom_group=np.array([0], np.int32),
                             group_h0=np.array([c["h0"]], np.float32))
        S = _eval(x, m, h, prob, np.array([[c["theta"]]], np.float32))
        assert abs(S[0, 0] - c["expect"]) <= 1e-6, c["name"]


def test_cmp_full_size_all_domains():
    """The 48-trace x 500-sample CMP gather, every domain, 32 random C each."""
    wl = configs.cmp_search(0)
    theta = random_theta(wl.problem.n_dom, 32, wl.de.lo, wl.de.hi, 1)
    S = _eval(wl.traces, wl.mid, wl.off, wl.problem, theta)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, theta)
    assert np.max(np.abs(S - ref)) <= TOL
    assert np.all((S >= 0) & (S <= 1 + 1e-6))


@pytest.mark.parametrize("P", [1, 4, 20, 37, 64])
def test_crs_small_line_ragged(P):
    """12 CMPs x 200 samples, apertures clipped at the line ends (uneven N),
    P not a multiple of the warp (a ragged tail of (domain, individual) pairs)."""
    wl = small_line(2)
    prob = wl.problem
    theta = random_theta(prob.n_dom, P, wl.de.lo, wl.de.hi, P)
    S = _eval(wl.traces, wl.mid, wl.off, prob, theta)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - ref)) <= TOL


@pytest.mark.parametrize("w", list(range(0, 9)))
def test_every_half_window(w):
    wl = small_line(3, n_cmp=5, ns=120, ap_half=2)
    prob = wl.problem
    prob.half_window = w
    theta = random_theta(prob.n_dom, 8, wl.de.lo, wl.de.hi, 10 + w)
    S = _eval(wl.traces, wl.mid, wl.off, prob, theta)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - ref)) <= TOL


def test_edge_cases_empty_zero_negative_beyond():
    """Empty aperture (N = 0), all-zero traces, T < 0 traces, windows past the
    end of the record, it0 = 0 and the last sample."""
    rng = np.random.default_rng(5)
    ns = 64
    x = rng.standard_normal((6, ns)).astype(np.float32)
    x[2] = 0.0
    mid = np.array([0, 10, 20, -10, -20, 0], np.float32)
    off = np.array([0, 100, 200, 300, 400, 2000], np.float32)
    prob = synth.Problem(op=1, half_window=5,
                         group_m0=np.array([0, 0, 5], np.float32),
                         group_dt=np.array([0.004, 0.004, 0.002], np.float32),
                         ap_ptr=np.array([0, 0, 1, 6], np.int32),
                         ap_idx=np.array([2, 0, 1, 2, 3, 4], np.int32),
                         dom_it0=np.array([3, 0, 63, 0, 10, 63, 40], np.int32),
                         dom_group=np.array([0, 1, 1, 2, 2, 2, 2], np.int32))
    theta = np.zeros((7, 5, 3), np.float32)
    theta[:, 0] = [0, 0, 1e-7]
    theta[:, 1] = [0, -1e-3, 0]          # T < 0 at |dm| = 10..20
    theta[:, 2] = [0, 0, 5e-6]           # far beyond the record
    theta[:, 3] = [3e-3, 0, 0]           # strong dip
    theta[:, 4] = [-6e-4, 1.5e-7, 5e-7]
    S = _eval(x, mid, off, prob, theta)
    ref = oracle.semblance.semblance_many(x, mid, off, prob, theta)
    assert np.max(np.abs(S - ref)) <= TOL
    assert np.all(S[0] == 0.0)           # empty aperture
    assert np.all(S[:, 2][[1, 2]] == 0.0)  # window beyond the record


def test_bf16_storage():
    wl = small_line(4)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 16, wl.de.lo, wl.de.hi, 4)
    S = _eval(wl.traces, wl.mid, wl.off, prob, theta, storage="bf16")
    ref_b = oracle.semblance.semblance_many(bf16_round(wl.traces), wl.mid, wl.off, prob, theta)
    ref_f = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - ref_b)) <= TOL
    assert np.max(np.abs(S - ref_f)) <= 2e-3


def test_reload_traces_host_and_device():
    wl = small_line(6, n_cmp=4, ns=100, ap_half=1)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 8, wl.de.lo, wl.de.hi, 6)
    other = np.flip(wl.traces, axis=0).copy()
    for storage in ("f32", "bf16"):
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, storage=storage,
                               device=dev())
        tt.tt_ctx_load_traces(ctx, torch.from_numpy(other).pin_memory())
        S1 = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
        tt.tt_ctx_load_traces(ctx, to_dev(wl.traces))
        S2 = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
        ctx.close()
        src1 = other if storage == "f32" else bf16_round(other)
        src2 = wl.traces if storage == "f32" else bf16_round(wl.traces)
        assert np.max(np.abs(S1 - oracle.semblance.semblance_many(
            src1, wl.mid, wl.off, prob, theta))) <= TOL
        assert np.max(np.abs(S2 - oracle.semblance.semblance_many(
            src2, wl.mid, wl.off, prob, theta))) <= TOL


def test_invalid_problem_rejected_on_device():
    wl = small_line(7, n_cmp=3, ns=60, ap_half=1)
    prob = wl.problem
    bad = synth.Problem(**{**prob.__dict__})
    bad.ap_idx = prob.ap_idx.copy()
    bad.ap_idx[3] = wl.traces.shape[0] + 5
    with pytest.raises(tt.TTError, match="ap_idx"):
        tt.tt_ctx_create(wl.traces, wl.mid, wl.off, bad, None, device=dev())
    bad = synth.Problem(**{**prob.__dict__})
    bad.dom_group = prob.dom_group.copy()
    bad.dom_group[-1] = 99
    with pytest.raises(tt.TTError, match="dom_group"):
        tt.tt_ctx_create(wl.traces, wl.mid, wl.off, bad, None, device=dev())
    bad = synth.Problem(**{**prob.__dict__})
    bad.group_dt = np.zeros_like(prob.group_dt)
    with pytest.raises(tt.TTError, match="group_dt"):
        tt.tt_ctx_create(wl.traces, wl.mid, wl.off, bad, None, device=dev())


@pytest.mark.slow
def test_full_line_sampled_outputs():
    """The 200-CMP x 48 x 1500 line at full size, NP = 64 random vectors at
    every domain (the launch the search makes each generation); a seeded
    sample of outputs is recomputed by the oracle, all lie in [0, 1]."""
    wl = configs.crs_line(0)
    prob = wl.problem
    rng = np.random.default_rng(9)
    theta_t = torch.empty((prob.n_dom, 64, 3), dtype=torch.float32, device=dev())
    lo = torch.tensor(wl.de.lo, device=dev())
    hi = torch.tensor(wl.de.hi, device=dev())
    g = torch.Generator(device=dev()).manual_seed(9)
    theta_t.copy_(lo + torch.rand(theta_t.shape, generator=g, device=dev()) * (hi - lo))
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, device=dev())
    tt.tt_ctx_autotune(ctx, theta_t)  # the bench's launch configuration
    S = tt.tt_semblance_eval(ctx, theta_t).cpu().numpy()
    ctx.close()
    theta = theta_t.cpu().numpy()
    assert np.all((S >= 0) & (S <= 1 + 1e-6))
    doms = rng.choice(prob.n_dom, 300, replace=False)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta[doms],
                                          domains=doms)
    assert np.max(np.abs(S[doms] - ref)) <= TOL
