"""FO-CRS operator (TT_OP_FOCRS, five parameters on a common-offset section)
on the GPU against the oracle.

* Semblance at random parameters on a small section (ragged apertures at the
  line ends): every kernel variant bit-identical, each within 1e-5 of the
  FP64 oracle, the small-launch split form too; BF16-stored traces within
  1e-5 of the oracle on the BF16-rounded record; long records (moveout
  form of the position) within 1e-5.
* Adjoint gradient against the FP64 oracle gradient in all five directions.
* The stacked output at random parameters.
* The whole search (DE + exchange + polish): S of the reported parameters
  reproduced by the oracle within 1e-5 except where a trace's T lies within
  FP32 rounding of 0 (the curvature terms of FO-CRS make T cross zero in the
  aperture; FP32 and FP64 may then disagree on T < 0, a discontinuity of S),
  call counts, and recovery of the two slopes and the Bmh, Bhh curvatures
  at event-centred samples of isolated strong events; the ENS sweep on the same section (call counts, S
  consistency).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from paper_2304_11399_gb300 import _lib
from gpu_util import dev, random_theta, to_dev, bf16_round, synth, configs

pytestmark = pytest.mark.gpu
TOL = 1e-5
VARIANTS = _lib.TUNE_CANDIDATES


def _sign_ambiguous(wl, theta_dom, doms):
    """Domains with an aperture trace whose T is within FP32 rounding of 0
    (|T| <= 1e-6 of the sum of its terms' magnitudes): FP32 and FP64 may take
    opposite sides of T < 0 there, reading zeros on one side and the record
    near sample 0 on the other, so their S may differ beyond 1e-5."""
    out = []
    for r, d in enumerate(doms):
        x, dt, dm, dh, t0 = oracle.semblance.domain_data(wl.traces, wl.mid, wl.off, wl.problem, d)
        Am, Ah, Bmm, Bmh, Bhh = (float(v) for v in theta_dom[r])
        q = t0 + Am * dm + Ah * dh
        terms = q * q + np.abs(Bmm * dm * dm) + np.abs(Bmh * dm * dh) + np.abs(Bhh * dh * dh)
        T = oracle.semblance.traveltime_sq(oracle.semblance.FOCRS, theta_dom[r], t0, dm, dh)
        out.append(bool(np.any(np.abs(T) <= 1e-6 * terms)))
    return np.array(out)


def _panel(seed=0, **kw):
    kw.setdefault("n_cmp", 12)
    kw.setdefault("ns", 220)
    kw.setdefault("n_events", 4)
    kw.setdefault("tau_max", 0.7)
    return configs.fo_panel(seed, **kw)


@pytest.mark.parametrize("P", [1, 7, 64])
def test_variants_and_split_match_oracle(P):
    wl = _panel(1)
    prob = wl.problem
    theta = random_theta(prob.n_dom, P, wl.de.lo, wl.de.hi, P)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    th = to_dev(theta)
    out = {}
    for kern, block in VARIANTS:
        tt.tt_ctx_set_option(ctx, "kernel", kern)
        tt.tt_ctx_set_option(ctx, "block", block)
        tt.tt_ctx_set_option(ctx, "split", False)
        out[(kern, block)] = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    tt.tt_ctx_set_option(ctx, "split", True)
    split = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    ctx.close()
    base = out[VARIANTS[0]]
    for k, v in out.items():
        assert np.array_equal(v, base), k
    assert np.max(np.abs(base - ref)) <= TOL
    assert np.max(np.abs(split - ref)) <= TOL


@pytest.mark.slow
def test_full_panel_sampled_outputs():
    """The FO-CRS bench workload at full size (the h0 = 1000 m section of the
    200-CMP line: 300,000 domains, up to 697 traces each), NP = 64 random
    vectors at every domain in the launch configuration the bench times
    (autotuned variant): 300 sampled domains recomputed by the oracle; a
    pair beyond 1e-5 must be a T-sign decision at the rounding level."""
    wl = configs.fo_panel(0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    th = torch.empty((prob.n_dom, 64, 5), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, th)
    tt.tt_ctx_autotune(ctx, th)
    S = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    ctx.close()
    doms = np.sort(np.random.default_rng(7).choice(prob.n_dom, 300, replace=False))
    theta = th[torch.as_tensor(doms, device=dev())].cpu().numpy()
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta, domains=doms)
    bad = np.argwhere(np.abs(S[doms] - ref) > TOL)
    for r, p in bad:
        assert _sign_ambiguous(wl, theta[r, p][None], [doms[r]])[0], (doms[r], p)
    assert bad.shape[0] <= 0.001 * ref.size, bad.shape


def test_bf16_storage_and_long_records():
    wl = _panel(2)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 8, wl.de.lo, wl.de.hi, 2)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, storage="bf16", device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    ref = oracle.semblance.semblance_many(bf16_round(wl.traces), wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - ref)) <= TOL
    # 2100 samples at 4 ms: u beyond 2048 samples takes the moveout form
    wl = _panel(3, n_cmp=6, ns=2100, n_events=5, tau_max=7.5, t0_range=(1500, 2100))
    prob = wl.problem
    theta = random_theta(prob.n_dom, 4, wl.de.lo, wl.de.hi, 3)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    assert np.max(np.abs(S - ref)) <= TOL


def test_gradient_matches_fp64_oracle():
    wl = _panel(4)
    prob = wl.problem
    rng = np.random.default_rng(4)
    doms = rng.choice(prob.n_dom, 400, replace=False)
    theta = random_theta(prob.n_dom, 1, wl.de.lo, wl.de.hi, 4)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, device=dev())
    S, G = tt.tt_semblance_grad(ctx, to_dev(theta))
    ctx.close()
    S, G = S.cpu().numpy()[doms, 0], G.cpu().numpy()[doms, 0]
    rS, rG = oracle.semblance.semblance_grad_many(wl.traces, wl.mid, wl.off, prob,
                                                  theta[doms], domains=doms)
    assert np.max(np.abs(S - rS[:, 0])) <= TOL
    rG = rG[:, 0]
    scale = np.median(np.abs(rG), axis=0) + 1e-30
    rel = np.abs(G - rG) / (np.abs(rG) + scale)
    assert np.quantile(rel, 0.99, axis=0).max() <= 2e-3, np.quantile(rel, 0.99, axis=0)


def test_stack_matches_oracle():
    wl = _panel(5)
    prob = wl.problem
    theta = random_theta(prob.n_dom, 1, wl.de.lo, wl.de.hi, 5)[:, 0]
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, device=dev())
    out = tt.tt_stack(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    ref = oracle.stack.stack_many(wl.traces, wl.mid, wl.off, prob, theta)
    step = float(np.max(np.abs(np.diff(wl.traces, axis=1))))
    tol = 4e-7 * (wl.traces.shape[1] + 5) * step + 1e-5 * step + \
        2e-6 * float(np.max(np.abs(wl.traces)))
    assert np.max(np.abs(out - ref)) <= tol


def test_search_recovers_slopes_and_ens_runs():
    wl = _panel(6, n_cmp=16, ns=300, n_events=4, snr=8.0, tau_max=1.0, np_=64, ng=100,
                exch_every=10, polish_steps=3)
    prob, line = wl.problem, wl.line
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    bt, bs, n = tt.tt_search(ctx)
    bt, bs = bt.cpu().numpy(), bs.cpu().numpy()
    edges = 2 * (prob.n_m0 * (prob.n_t0 - 1) + prob.n_t0 * (prob.n_m0 - 1))
    assert n == oracle.counts.search_calls(prob.n_dom, 64, 100, 10 * edges, 3)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, bt[:, None, :])[:, 0]
    bad = np.nonzero(np.abs(ref - bs) > TOL)[0]
    # every excess is a T-sign decision at the rounding level, and rare
    assert np.all(_sign_ambiguous(wl, bt[bad], bad)) and bad.size <= 0.001 * prob.n_dom, bad
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    hits = tried = 0
    for e, ev in enumerate(line.events):
        others = np.delete(line.events[:, 1], e)
        if not (np.all(np.abs(others - ev[1]) > 0.1) and abs(ev[5]) > 0.6):
            continue
        for c in range(3, line.n_cmp - 3):
            p = synth.gathers.fo_recentre(ev, line.cmp_x[c], 1000.0)
            if p is None or abs(line.cmp_x[c] - ev[0]) > 40:
                continue
            it0 = int(round(p[0] / line.dt))
            if not 10 <= it0 < line.ns - 10:
                continue
            d = c * prob.n_t0 + it0
            tried += 1
            # slopes and the offset curvatures; Bmm is weakly constrained by the
            # +-100 m midpoint aperture
            ok = all(abs(bt[d, k] - p[1 + k]) <= 0.01 * (hi[k] - lo[k]) for k in (0, 1, 3, 4))
            hits += int(ok)
    assert tried >= 4 and hits >= 0.75 * tried, (hits, tried)
    # the paper's ENS sweep on the same section
    th, S, n_e = tt.tt_ens_search(ctx, 5, 1, 5, 1, 2, 1, 8)
    ctx.close()
    assert n_e == oracle.counts.ens_calls(prob.n_dom, 5, 1, 5, 1, 2, 1)
    th = th.cpu().numpy()
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, th[:, None, :])[:, 0]
    bad = np.nonzero(np.abs(ref - S.cpu().numpy()) > TOL)[0]
    assert np.all(_sign_ambiguous(wl, th[bad], bad)) and bad.size <= 0.001 * prob.n_dom, bad
