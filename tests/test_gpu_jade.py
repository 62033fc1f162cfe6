"""JADE adaptation (cfg.adapt = 1) on the GPU against the oracle.

Step level: the kernel and ``oracle.jade`` are fed the same fitness arrays
for a run of generations (fused select + mutate steps, a select-only step
as before an exchange, a mutate-only step after it). The F_i / CR_i draws,
the archive and the memory are internal state, so they are compared through
their effect: every population, fitness, best index and trial must match
bit for bit, generation after generation. NP = 8 fills the archive within
two generations and exercises its random replacement; NP = 37 and 64 span
two 32-member chunks of the warp-level selection.

Search level: the adaptive tt_search is deterministic, equal under graph
replay and eager launching, reports S that the oracle reproduces within
1e-5, and recovers the CMP gather's velocities.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import jade
import paper_2304_11399_gb300 as tt
from gpu_util import dev, to_dev, small_line, configs

pytestmark = pytest.mark.gpu
f32 = np.float32


def _ctx(NP, op, seed, F0=0.5, CR0=0.5):
    wl = small_line(0, n_cmp=3, ns=27, ap_half=1, np_=NP, t0_range=(10, 17))
    wl.de.seed, wl.de.F, wl.de.CR, wl.de.adapt = seed, F0, CR0, 1
    if op == 0:
        wl.problem.op = 0
        wl.de.lo, wl.de.hi = (configs.C_BOUNDS_CMP[0],), (configs.C_BOUNDS_CMP[1],)
    return tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev()), wl


def _trial_fit(rng, fit):
    """Children that are strictly better for ~60% of members, equal for a
    few, worse or NaN for the rest."""
    base = np.where(np.isnan(fit), 0.0, fit)
    u = rng.uniform(0, 1, fit.shape)
    t = np.where(u < 0.6, base + rng.uniform(1e-3, 0.2, fit.shape),
                 base - rng.uniform(1e-3, 0.2, fit.shape)).astype(f32)
    t[u > 0.95] = fit[u > 0.95]      # ties: taken but no success
    t[(u > 0.9) & (u <= 0.92)] = np.nan
    return t


@pytest.mark.parametrize("op,NP,seed,F0,CR0", [(1, 8, 3, 0.5, 0.5), (1, 37, 2, 0.3, 0.9),
                                               (0, 16, 11, 0.5, 0.5),
                                               (1, 64, 2 ** 40 + 7, 0.8, 0.1)])
def test_generations_bit_exact(op, NP, seed, F0, CR0):
    ctx, wl = _ctx(NP, op, seed, F0, CR0)
    n, D = ctx.n_dom, ctx.D
    lo, hi = np.array(wl.de.lo, f32), np.array(wl.de.hi, f32)
    rng = np.random.default_rng(seed % 997)
    p_t = torch.empty((n, NP, D), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, p_t)
    pop = oracle.de.de_step(0, np.zeros((n, NP, D), f32), None, None, None, seed, F0, CR0,
                            lo, hi)[0]
    np.testing.assert_array_equal(p_t.cpu().numpy(), pop)
    fit = rng.uniform(0, 1, (n, NP)).astype(f32)
    fit[0, 1] = np.nan
    f_t = to_dev(fit)
    st = [jade.new_state(NP, D, F0, CR0) for _ in range(n)]
    best = torch.empty((n,), dtype=torch.int32, device=dev())

    def check(nxt=None, rtrial=None, rbest=None):
        np.testing.assert_array_equal(p_t.cpu().numpy(), pop)
        np.testing.assert_array_equal(f_t.cpu().numpy(), fit)
        if nxt is not None:
            np.testing.assert_array_equal(best.cpu().numpy(), rbest)
            np.testing.assert_array_equal(nxt.cpu().numpy(), rtrial)

    def ora_select(g_trial, trial, tfit):
        for d in range(n):
            pop[d], fit[d] = jade.select_adapt(st[d], seed, d, g_trial, pop[d], fit[d],
                                               trial[d], tfit[d])

    def ora_mutate(g):
        trial = np.empty_like(pop)
        b = np.empty(n, np.int32)
        for d in range(n):
            trial[d], b[d] = jade.trial_population(st[d], seed, d, g, pop[d], fit[d], lo, hi)
        return trial, b

    pending = None     # (trial, tfit, generation) awaiting selection
    for g in range(1, 11):
        nxt = torch.empty_like(p_t)
        if pending is None:
            tt.tt_de_step(ctx, g, p_t, f_t, None, None, nxt, best)
        else:
            tt.tt_de_step(ctx, g, p_t, f_t, to_dev(pending[0]), to_dev(pending[1]), nxt, best)
            ora_select(pending[2], pending[0], pending[1])
        rtrial, rb = ora_mutate(g)
        check(nxt, rtrial, rb)
        pending = (rtrial, _trial_fit(rng, fit), g)
        if g in (4, 10):   # select-only, as before an exchange and at the end
            tt.tt_de_step(ctx, g, p_t, f_t, to_dev(pending[0]), to_dev(pending[1]))
            ora_select(g, pending[0], pending[1])
            check()
            pending = None
    assert any(s.n_arc == NP for s in st)
    assert len({(float(s.mu_f), float(s.mu_cr)) for s in st}) > 1
    ctx.close()


def test_adaptive_search_deterministic_graph_and_oracle_consistent():
    wl = configs.crs_line(3, n_cmp=6, ns=160, n_events=2, ap_half=2, np_=24, ng=20,
                          exch_every=5, polish_steps=2, tau_max=0.5)
    wl.de.adapt = 1
    prob = wl.problem
    out = []
    for graph in (False, True, True):
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
        tt.tt_ctx_set_option(ctx, "search_graph", graph)
        bt, bs, n = tt.tt_search(ctx)
        out.append((bt.cpu().numpy(), bs.cpu().numpy(), n))
        ctx.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o[0], out[0][0])
        np.testing.assert_array_equal(o[1], out[0][1])
        assert o[2] == out[0][2]
    bt, bs, n = out[0]
    n_m0, n_t0 = prob.n_m0, prob.n_t0
    edges = 2 * (n_m0 * (n_t0 - 1) + n_t0 * (n_m0 - 1))
    assert n == oracle.counts.search_calls(prob.n_dom, 24, 20, 4 * edges, 2)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, bt[:, None, :])[:, 0]
    assert np.max(np.abs(ref - bs)) <= 1e-5


def test_adaptive_cmp_search_recovers_velocities():
    wl = configs.cmp_search(0)
    wl.de.adapt, wl.de.F, wl.de.CR = 1, 0.5, 0.5
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    bt, bs, n = tt.tt_search(ctx)
    bt = bt.cpu().numpy()
    ctx.close()
    hits = tried = 0
    for e in range(len(wl.line.events)):
        ev = wl.line.events[e]
        others = np.delete(wl.line.events[:, 1], e)
        if not (np.all(np.abs(others - ev[1]) > 12 * wl.dt) and abs(ev[5]) > 0.6):
            continue
        it0 = int(round(ev[1] / wl.dt))
        tried += 1
        hits += int(abs(bt[it0, 0] - ev[4]) <= 0.01 * ev[4])
    assert tried >= 3 and hits == tried


def test_invalid_adaptive_settings_rejected():
    wl = small_line(0, n_cmp=3, ns=27, ap_half=1, np_=8, t0_range=(10, 17))
    wl.de.adapt, wl.de.F = 1, 1.5
    with pytest.raises(tt.TTError, match="initial F"):
        tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    wl.de.adapt, wl.de.F = 2, 0.5
    with pytest.raises(tt.TTError, match="adapt"):
        tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
