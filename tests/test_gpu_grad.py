"""GPU adjoint gradient (tt_semblance_grad) and the autograd wrapper.

On the 48-trace CMP gather, 1000 random (m0, t0, theta) points of the CRS
operator (m0 off the gather's midpoint so that A and B matter) are checked
against the oracle's FP64 analytic gradient and against central finite
differences with h = 1e-4 of max(|theta_d|, range_d). The gradient jumps
where a trace's position crosses a sample (the interpolation kinks), so
points with a trace within 1e-3 samples of a kink (or, for FD, crossing one
within +-h) are excluded, as decided in FP64 on the evaluated parameters.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, to_dev, configs

pytestmark = pytest.mark.gpu


def _positions(wl, prob, theta, d):
    x, dt, dm, h, t0 = oracle.semblance.domain_data(wl.traces, wl.mid, wl.off, prob, d)
    T = oracle.semblance.traveltime_sq(prob.op, theta.astype(np.float64), t0, dm, h)
    return np.sqrt(np.maximum(T, 0.0)) / dt, T


@pytest.fixture(scope="module")
def points():
    wl = configs.cmp_search(0)
    prob, theta = configs.random_points(wl.line, 1000, seed=4)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, device=dev())
    S, G = tt.tt_semblance_grad(ctx, to_dev(theta))
    S, G = S.cpu().numpy()[:, 0], G.cpu().numpy()[:, 0]
    yield wl, prob, theta, S, G, ctx
    ctx.close()


def test_grad_matches_fp64_oracle(points):
    wl, prob, theta, S, G = points[:5]
    rS, rG = oracle.semblance.semblance_grad_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - rS[:, 0])) <= 1e-5
    scale = np.median(np.abs(rG[:, 0]), axis=0) + 1e-30
    used = 0
    for d in range(prob.n_dom):
        u, T = _positions(wl, prob, theta[d, 0], d)
        fr = u - np.floor(u)
        if np.any((T > 0) & ((fr < 1e-3) | (fr > 1 - 1e-3))):
            continue
        used += 1
        err = np.abs(G[d] - rG[d, 0]) / (np.abs(rG[d, 0]) + scale)
        assert np.all(err <= 2e-3), (d, G[d], rG[d, 0])
    assert used >= 800


def test_grad_matches_central_differences(points):
    wl, prob, theta, S, G, ctx = points
    lo, hi = np.array(configs.CRS_LO), np.array(configs.CRS_HI)
    n = prob.n_dom
    h = 1e-4 * np.maximum(np.abs(theta[:, 0, :]), hi - lo)
    checked = checked32 = 0
    for k in range(3):
        tp, tm = theta.copy(), theta.copy()
        tp[:, 0, k] += h[:, k].astype(np.float32)
        tm[:, 0, k] -= h[:, k].astype(np.float32)
        hk = (tp[:, 0, k].astype(np.float64) - tm[:, 0, k].astype(np.float64)) / 2
        Sp = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, tp)[:, 0]
        Sm = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, tm)[:, 0]
        Sp_g = tt.tt_semblance_eval(ctx, to_dev(tp)).cpu().numpy()[:, 0]
        Sm_g = tt.tt_semblance_eval(ctx, to_dev(tm)).cpu().numpy()[:, 0]
        fd64 = (Sp - Sm) / (2 * hk)
        fd32 = (Sp_g.astype(np.float64) - Sm_g) / (2 * hk)
        scale = np.median(np.abs(fd64)) + 1e-30
        for d in range(n):
            u0, T0 = _positions(wl, prob, theta[d, 0], d)
            fr = u0 - np.floor(u0)
            if np.any((T0 > 0) & ((fr < 1e-3) | (fr > 1 - 1e-3))):
                continue  # a trace at a kink: FP32 and FP64 may take opposite sides
            up, Tp = _positions(wl, prob, tp[d, 0], d)
            um, Tm = _positions(wl, prob, tm[d, 0], d)
            if np.any(np.floor(up) != np.floor(um)) or np.any((Tp > 0) != (Tm > 0)):
                continue
            checked += 1
            assert abs(G[d, k] - fd64[d]) <= 2e-2 * (abs(fd64[d]) + scale), (k, d)
            # the FP32 difference quotient carries the rounding of two FP32
            # semblance values (observed up to ~1e-6 each) divided by 2h, so it
            # is checked only where the change of S resolves the gradient
            if abs(fd64[d]) * 2 * hk[d] >= 2e-5:
                noise = 2e-6 / (2 * hk[d])
                assert abs(G[d, k] - fd32[d]) <= 5e-2 * (abs(fd64[d]) + scale) + noise, (k, d)
                checked32 += 1
    assert checked >= 600 and checked32 >= 300


def test_autograd_backward_is_adjoint(points):
    wl, prob, theta, S, G, ctx = points
    th = to_dev(theta).requires_grad_(True)
    out = tt.semblance(ctx, th)
    w = torch.linspace(0.5, 1.5, out.numel(), device=dev()).reshape(out.shape)
    (out * w).sum().backward()
    expect = w.unsqueeze(-1) * to_dev(G).unsqueeze(1)
    torch.testing.assert_close(th.grad, expect, rtol=1e-6, atol=0)
    # the forward is K1 (at 1000 points the aperture-split small-launch
    # kernel), S is K2's: two FP32 summation orders of the same sums
    np.testing.assert_allclose(out.detach().cpu().numpy()[:, 0], S, rtol=0, atol=1e-6)


def test_cmp_gradient_and_polish():
    """CMP operator (D = 1) gradient on the gather, and tt_polish never
    lowering S from perturbed starts near each isolated event."""
    wl = configs.cmp_search(0, polish_steps=5)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    rng = np.random.default_rng(2)
    theta = (wl.de.lo[0] + rng.uniform(0, 1, (prob.n_dom, 1, 1)) *
             (wl.de.hi[0] - wl.de.lo[0])).astype(np.float32)
    S, G = tt.tt_semblance_grad(ctx, to_dev(theta))
    rS, rG = oracle.semblance.semblance_grad_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S.cpu().numpy() - rS)) <= 1e-5
    g, r = G.cpu().numpy()[:, 0, 0], rG[:, 0, 0]
    scale = np.median(np.abs(r))
    assert np.quantile(np.abs(g - r) / (np.abs(r) + scale), 0.99) <= 2e-3
    start = theta[:, 0, :].copy()
    for e in range(len(wl.line.events)):
        it0 = int(round(wl.line.events[e, 1] / wl.dt))
        start[it0, 0] = wl.line.events[e, 4] * 1.01
    th = to_dev(start)
    S0 = tt.tt_semblance_eval(ctx, th[:, None, :].contiguous()).cpu().numpy()[:, 0]
    th, Sp = tt.tt_polish(ctx, th, 5, wl.de.polish_lr)
    Sp = Sp.cpu().numpy()
    # iterate 0's S comes from K2, S0 from K1 (two FP32 summation orders)
    assert np.all(Sp >= S0 - 1e-6)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob,
                                          th.cpu().numpy()[:, None, :])[:, 0]
    assert np.max(np.abs(ref - Sp)) <= 1e-5
    ctx.close()
