"""Large-line workload with BF16-stored traces: a central slab of the
2000-CMP x 120-offset x 2000-sample line (2 ms), aperture +-25 CMPs (N up to
6120 traces per semblance call), NP = 96.

BF16 storage rounds the record once; the arithmetic is FP32 with the energy
summed in FP64 over 32-trace chunks. Bars: |dS| <= 1e-5 against the oracle
on the same BF16-rounded record (the kernel's arithmetic), <= 2e-3 against
the oracle on the FP32 record (the storage precision).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, random_theta, to_dev, bf16_round, synth, configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab():
    wl = configs.large_line(0, n_cmp=60, n_events=4, ng=120)
    return wl


def test_bf16_long_aperture_parity(slab):
    wl = slab
    prob = synth.line_problem(wl.line, half_window=5, ap_half=25, cmps=list(range(25, 35)),
                              t0_range=(0, 2000))
    theta = random_theta(prob.n_dom, 96, wl.de.lo, wl.de.hi, 5)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, None, storage="bf16", device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    ctx.close()
    assert np.all((S >= 0) & (S <= 1 + 1e-6))
    rng = np.random.default_rng(1)
    doms = rng.choice(prob.n_dom, 40, replace=False)
    xb = bf16_round(wl.traces)
    ref_b = oracle.semblance.semblance_many(xb, wl.mid, wl.off, prob, theta[doms], domains=doms)
    ref_f = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta[doms],
                                            domains=doms)
    assert np.max(np.abs(S[doms] - ref_b)) <= 1e-5
    assert np.max(np.abs(S[doms] - ref_f)) <= 2e-3


def test_bf16_slab_search(slab):
    """Full settings (NP 96, NG 120, exchange every 10, 5 polish steps) on 4
    central CMPs x 2000 samples; the reported S of a 1% sample of the domains
    is re-evaluated by the oracle (BF16-rounded record <= 1e-5, FP32 record
    <= 2e-3) and recovery is checked at the events' zero-offset times."""
    wl = slab
    cm = list(range(28, 32))
    prob = synth.line_problem(wl.line, half_window=5, ap_half=25, cmps=cm, t0_range=(0, 2000))
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, storage="bf16", device=dev())
    bt, bs, n = tt.tt_search(ctx)
    bt, bs = bt.cpu().numpy(), bs.cpu().numpy()
    ctx.close()
    edges = 2 * (prob.n_m0 * (prob.n_t0 - 1) + prob.n_t0 * (prob.n_m0 - 1))
    assert n == oracle.counts.search_calls(prob.n_dom, 96, 120, 12 * edges, 5)
    rng = np.random.default_rng(2)
    doms = rng.choice(prob.n_dom, prob.n_dom // 100, replace=False)
    ref_b = oracle.semblance.semblance_many(bf16_round(wl.traces), wl.mid, wl.off, prob,
                                            bt[doms][:, None, :], domains=doms)[:, 0]
    ref_f = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob,
                                            bt[doms][:, None, :], domains=doms)[:, 0]
    assert np.max(np.abs(ref_b - bs[doms])) <= 1e-5
    assert np.max(np.abs(ref_f - bs[doms])) <= 2e-3
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    tried = hits = 0
    for ev in wl.line.events:
        for ci, c in enumerate(cm):
            truth = synth.crs_recentre(ev, wl.line.cmp_x[c])
            if truth is None or abs(ev[5]) < 0.7:
                continue
            it = int(round(truth[0] / wl.dt))
            if not (40 <= it < 1960 and lo[0] < truth[1] < hi[0] and lo[2] < truth[3] < hi[2]):
                continue
            d = ci * prob.n_t0 + it
            tried += 1
            hits += int(abs(bt[d, 0] - truth[1]) <= 0.01 * (hi[0] - lo[0])
                        and abs(bt[d, 2] - truth[3]) <= 0.01 * truth[3])
    assert tried >= 4 and hits >= 0.75 * tried, (hits, tried)


@pytest.mark.slow
def test_bench_slab_sampled_outputs():
    """The bench's large-line case: the central 100-CMP slab of the full
    2000-CMP line (BF16-stored, aperture +-25 CMPs), NP = 96 random vectors
    at every domain, autotuned variant; 200 sampled domains recomputed by the
    oracle on the BF16-rounded record."""
    wl = configs.large_line(0, cmps=list(range(950, 1050)))
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, storage="bf16", device=dev())
    th = torch.empty((prob.n_dom, 96, 3), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, th)
    tt.tt_ctx_autotune(ctx, th)
    S = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    ctx.close()
    doms = np.sort(np.random.default_rng(6).choice(prob.n_dom, 200, replace=False))
    theta = th[torch.as_tensor(doms, device=dev())].cpu().numpy()
    idx = np.unique(prob.ap_idx)
    rounded = wl.traces.copy()
    rounded[idx] = bf16_round(wl.traces[idx])
    ref = oracle.semblance.semblance_many(rounded, wl.mid, wl.off, prob, theta, domains=doms)
    assert np.max(np.abs(S[doms] - ref)) <= 1e-5


@pytest.mark.slow
def test_whole_line_one_launch_sampled_outputs():
    """The largest configuration in one launch: all 4,000,000 domains of the
    2000-CMP BF16 line (up to 6120 traces each), NP = 96 random vectors,
    384M pairs and 2.3e12 trace evaluations; 100 sampled domains recomputed
    by the oracle on the BF16-rounded record."""
    wl = configs.large_line(0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, storage="bf16", device=dev())
    th = torch.empty((prob.n_dom, 96, 3), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, th)
    S = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    ctx.close()
    assert np.all((S >= 0) & (S <= 1 + 1e-6))
    doms = np.sort(np.random.default_rng(9).choice(prob.n_dom, 100, replace=False))
    theta = th[torch.as_tensor(doms, device=dev())].cpu().numpy()
    del th
    idx = np.unique(np.concatenate([prob.ap_idx[prob.ap_ptr[g]:prob.ap_ptr[g + 1]]
                                    for g in np.unique(prob.dom_group[doms])]))
    rounded = np.zeros_like(wl.traces)
    rounded[idx] = bf16_round(wl.traces[idx])
    ref = oracle.semblance.semblance_many(rounded, wl.mid, wl.off, prob, theta, domains=doms)
    assert np.max(np.abs(S[doms] - ref)) <= 1e-5
