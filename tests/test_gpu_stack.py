"""Stacked zero-offset output (tt_stack) on the GPU against the oracle.

Tolerance, derived from the arithmetic: the kernel sums FP32 amplitudes (a
32-lane butterfly over per-lane sums; relative error below 1e-6 of the sum
of |a| for the apertures here) at FP32 positions. A position is off by at
most 4e-7 u samples (approximate square root plus the rounding of T) in the
direct form, 1e-5 samples in the moveout form, and moves a linearly
interpolated amplitude by at most that times the largest step between two
adjacent samples of the record. So, per test,
    |out - stack| <= 4e-7 u_max max|dx| + 1e-5 max|dx| + 2e-6 max|x|.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, random_theta, to_dev, bf16_round, small_line, synth, configs

pytestmark = pytest.mark.gpu


def _tol(x, umax):
    x = np.asarray(x, np.float64)
    step = float(np.max(np.abs(np.diff(x, axis=1)))) if x.shape[1] > 1 else 0.0
    return 4e-7 * umax * step + 1e-5 * step + 2e-6 * float(np.max(np.abs(x)))


def _stack(traces, mid, off, prob, theta, storage="f32", ctx_out=False):
    ctx = tt.tt_ctx_create(traces, mid, off, prob, None, storage=storage, device=dev())
    out = tt.tt_stack(ctx, to_dev(theta)).cpu().numpy()
    again = tt.tt_stack(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    assert np.array_equal(out, again)  # fixed summation order
    return out


def test_hand_worked_stacks_through_cabi(golden_dir):
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
        out = _stack(x, m, h, prob, np.array([c["theta"]], np.float32))
        assert abs(out[0] - c["stack"]) <= 1e-6, c["name"]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_small_line_ragged_apertures(storage):
    """12 CMPs x 200 samples, apertures clipped at the line ends."""
    wl = small_line(41)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 1, wl.de.lo, wl.de.hi, 41)[:, 0]
    out = _stack(wl.traces, wl.mid, wl.off, prob, theta, storage)
    src = wl.traces if storage == "f32" else bf16_round(wl.traces)
    ref = oracle.stack.stack_many(src, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(out - ref)) <= _tol(src, wl.traces.shape[1] + 5)


def test_cmp_gather_at_every_sample():
    wl = configs.cmp_search(3)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 1, wl.de.lo, wl.de.hi, 3)[:, 0]
    out = _stack(wl.traces, wl.mid, wl.off, prob, theta)
    ref = oracle.stack.stack_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(out - ref)) <= _tol(wl.traces, wl.traces.shape[1] + 5)


def test_edge_cases_empty_negative_beyond():
    rng = np.random.default_rng(5)
    ns = 64
    x = rng.standard_normal((6, ns)).astype(np.float32)
    mid = np.array([0, 10, 20, -10, -20, 0], np.float32)
    off = np.array([0, 100, 200, 300, 400, 2000], np.float32)
    prob = synth.Problem(op=1, half_window=5,
                         group_m0=np.array([0, 0, 5], np.float32),
                         group_dt=np.array([0.004, 0.004, 0.002], np.float32),
                         ap_ptr=np.array([0, 0, 1, 6], np.int32),
                         ap_idx=np.array([2, 0, 1, 2, 3, 4], np.int32),
                         dom_it0=np.array([3, 0, 63, 0, 10, 63, 40], np.int32),
                         dom_group=np.array([0, 1, 1, 2, 2, 2, 2], np.int32))
    for th in ([0, 0, 1e-7], [0, -1e-3, 0], [0, 0, 5e-6], [3e-3, 0, 0], [-6e-4, 1.5e-7, 5e-7]):
        theta = np.tile(np.array(th, np.float32), (7, 1))
        out = _stack(x, mid, off, prob, theta)
        ref = oracle.stack.stack_many(x, mid, off, prob, theta)
        assert np.max(np.abs(out - ref)) <= _tol(x, ns + 5), th
        assert out[0] == 0.0  # empty aperture
    theta = np.tile(np.array([0, 0, 5e-6], np.float32), (7, 1))
    assert np.all(_stack(x, mid, off, prob, theta)[[1, 2]] == 0.0)  # past the record


def test_moveout_form_on_long_records():
    """3000 samples at 2 ms: positions take the moveout form."""
    wl = configs.large_line(2, n_cmp=12, ns=3000, n_events=4, ap_half=2, cmps=[5, 6],
                            t0_range=(0, 3000))
    prob = wl.problem
    theta = random_theta(prob.n_dom, 1, wl.de.lo, wl.de.hi, 2)[:, 0]
    out = _stack(wl.traces, wl.mid, wl.off, prob, theta)
    ref = oracle.stack.stack_many(wl.traces, wl.mid, wl.off, prob, theta)
    step = float(np.max(np.abs(np.diff(wl.traces, axis=1))))
    assert np.max(np.abs(out - ref)) <= 1e-5 * step + 2e-6 * float(np.max(np.abs(wl.traces)))


@pytest.mark.slow
def test_full_line_sampled_outputs_at_searched_parameters():
    """The 200-CMP x 48 x 1500 line at full size: stack at the parameters of a
    short search (the call sequence a user makes), sampled outputs recomputed
    by the oracle."""
    wl = configs.crs_line(0, ng=10, polish_steps=0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    th, S, _ = tt.tt_search(ctx)
    out = tt.tt_stack(ctx, th).cpu().numpy()
    ctx.close()
    theta = th.cpu().numpy()
    doms = np.random.default_rng(10).choice(prob.n_dom, 400, replace=False)
    ref = oracle.stack.stack_many(wl.traces, wl.mid, wl.off, prob, theta[doms], domains=doms)
    assert np.max(np.abs(out[doms] - ref)) <= _tol(wl.traces, wl.traces.shape[1] + 5)
