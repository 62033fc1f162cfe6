"""Pins of the oracle's exchange, eval counts and whole search."""
import os

import numpy as np
import pytest

from oracle import counts, de, exchange as ex, search as osearch
from oracle.semblance import semblance, semblance_many
import synth
from synth import configs

f32 = np.float32


# ----------------------------------------------------------------- counts

def test_eval_counts_match_paper(golden_dir):
    rows = {}
    for line in open(os.path.join(golden_dir, "eval_counts.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, P, NP, NG, e = line.split()
            rows[k] = (int(P), int(NP), int(NG), float(e))
    P, NP, NG, e = rows["jade_per_sample"]
    assert counts.jade_calls(P, NP, NG) == e
    P, NP, NG, e = rows["ens_per_sample"]
    assert counts.ens_calls(P, NP, NG, 5, 1, 2, 1) == e
    P, NP, NG, e = rows["jade_ds3"]
    assert round(counts.jade_calls(P, NP, NG) / 1e10, 1) == e / 1e10
    P, NP, NG, e = rows["ens_ds3"]
    assert round(counts.ens_calls(P, NP, NG, 5, 1, 2, 1) / 1e10, 1) == e / 1e10


def test_jade_over_ens_tends_to_nskip_plus_one():
    P = 3 * 10 ** 6
    r = [counts.jade_calls(P, n, n) / counts.ens_calls(P, n, n, 5, 1, 2, 1) for n in (20, 80, 400)]
    assert r[0] < r[1] < r[2] < 3.0
    assert r[2] == pytest.approx(3.0, abs=0.01)
    # ENS never costs more than JADE for NP_f >= 5, NG_f >= 1 (Sec. 6.1)
    for n in range(5, 40):
        for g in range(1, 40):
            assert counts.ens_calls(P, n, g, 5, 1, 2, 1) <= counts.jade_calls(P, n, g) * 1.14


# ----------------------------------------------------------------- exchange

def test_neighbours_grid():
    n_m0, n_t0 = 3, 4
    assert ex.neighbours(0, n_m0, n_t0) == [1, 4]
    assert ex.neighbours(3, n_m0, n_t0) == [2, 7]
    assert ex.neighbours(5, n_m0, n_t0) == [4, 6, 1, 9]
    assert ex.neighbours(11, n_m0, n_t0) == [10, 7]
    n = [len(ex.neighbours(d, n_m0, n_t0)) for d in range(12)]
    assert sum(n) == 2 * (n_m0 * (n_t0 - 1) + n_t0 * (n_m0 - 1))


def test_exchange_plan_slots_and_imports():
    n_m0, n_t0, NP, D = 2, 3, 6, 3
    rng = np.random.default_rng(0)
    pop = rng.uniform(-1, 1, (6, NP, D)).astype(f32)
    fit = np.array([[0.9, 0.1, 0.5, 0.1, 0.3, 0.2]] * 6, f32)
    fit[4] = [0.2, 0.2, 0.2, 0.2, 0.2, 0.2]  # all equal: best is 0, it is kept
    snap = ex.best_snapshot(pop, fit)
    np.testing.assert_array_equal(snap[0], pop[0, 0])
    imports, slots = ex.exchange_plan(n_m0, n_t0, pop, fit, snap)
    # domain 1 = (m0 0, t0 1): neighbours 0, 2, 4 -> worst slots 1, 3, 5
    assert list(slots[1]) == [1, 3, 5, -1]
    np.testing.assert_array_equal(imports[1, 0], snap[0])
    np.testing.assert_array_equal(imports[1, 2], snap[4])
    # domain 4 = (m0 1, t0 1): neighbours 3, 5, 1 ; all fit equal, best 0 excluded
    assert list(slots[4]) == [1, 2, 3, -1]
    for d in range(6):
        k = len(ex.neighbours(d, n_m0, n_t0))
        assert np.sum(slots[d] >= 0) == k
        assert de.best_index(fit[d]) not in slots[d]
    ifit = np.full((6, 4), 0.99, f32)
    p2, f2 = ex.apply_exchange(pop, fit, imports, slots, ifit)
    np.testing.assert_array_equal(p2[1, 5], snap[4])
    assert f2[1, 5] == f32(0.99) and f2[1, 0] == fit[1, 0]


# ----------------------------------------------------------------- search

def test_polish_never_lowers_and_improves_near_peak():
    wl = configs.cmp_search(0)
    x = wl.traces.astype(np.float64)
    ev = wl.line.events[0]
    it0 = int(round(ev[1] / wl.dt))
    t0 = it0 * wl.dt
    C = ev[4]
    lo, hi = wl.de.lo, wl.de.hi
    start = np.array([C * 1.02])
    S0 = semblance(x, wl.dt, np.zeros(48), wl.off, t0, 0, start, 5)
    th, S, n = osearch.polish_point(x, wl.dt, np.zeros(48), wl.off.astype(float), t0, 0, 5,
                                    start, lo, hi, 5, wl.de.polish_lr)
    assert n == 6
    assert S >= S0
    assert abs(th[0] - C) <= abs(start[0] - C)


def _event_domains(wl, ng_min_sep=12):
    """Zero-offset samples of the CMP events that are isolated in time."""
    ev = wl.line.events
    t = ev[:, 1]
    keep = []
    for e in range(len(ev)):
        others = np.delete(t, e)
        if np.all(np.abs(others - t[e]) > ng_min_sep * wl.dt) and abs(ev[e, 5]) > 0.6:
            keep.append(e)
    return keep


def test_cmp_search_recovers_generating_velocity():
    wl = configs.cmp_search(0, np_=32, ng=50)
    keep = _event_domains(wl)
    assert len(keep) >= 3
    ev = wl.line.events
    it0 = np.array([int(round(ev[e, 1] / wl.dt)) for e in keep], np.int32)
    prob = synth.cmp_problem(wl.line, half_window=5, it0=it0)
    th, S, n = osearch.search(wl.traces, wl.mid, wl.off, prob, wl.de)
    assert n == counts.search_calls(len(keep), 32, 50, 0, 0)
    for r, e in enumerate(keep):
        assert th[r, 0] == pytest.approx(ev[e, 4], rel=0.01), (e, th[r, 0], ev[e, 4])
        assert S[r] > 0.3


def test_crs_search_with_exchange_counts_and_recovery():
    """Small CRS line: the exchange count matches the grid and the search
    finds the recentred parameters of an isolated strong event."""
    wl = configs.crs_line(3, n_cmp=9, ns=300, n_events=1, ap_half=3, np_=24, ng=30,
                          exch_every=10, polish_steps=2, snr=20.0, tau_max=0.9)
    ev = wl.line.events[0]
    mid_cmp = 4
    m0 = wl.line.cmp_x[mid_cmp]
    truth = synth.crs_recentre(ev, m0)
    assert truth is not None
    it_c = int(round(truth[0] / wl.dt))
    prob = synth.line_problem(wl.line, half_window=5, ap_half=3, cmps=[3, 4, 5],
                              t0_range=(it_c - 2, it_c + 3))
    th, S, n = osearch.search(wl.traces, wl.mid, wl.off, prob, wl.de)
    n_edges = 2 * (3 * 4 + 5 * 2)
    assert n == counts.search_calls(15, 24, 30, 3 * n_edges, 2)
    d = 1 * 5 + 2  # centre CMP, centre sample
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    # A within 1% of its bound range, C within 1% (B is weakly constrained
    # over a +-3 CMP aperture and is checked only for sign-free closeness)
    assert abs(th[d, 0] - truth[1]) <= 0.01 * (hi[0] - lo[0])
    assert th[d, 2] == pytest.approx(truth[3], rel=0.01)
    assert S[d] > 0.5


def test_exchange_result_is_the_best_of_own_and_neighbours_bests():
    """With the exchange as the last step (NG = exch_every, no polish), every
    sample's result is the best of its own pre-exchange best and the
    neighbours' pre-exchange bests evaluated at it: the imports replace
    members other than the own best (Sec. 3.3). The pre-exchange bests are
    those of the same search without exchange (same draws up to that point).
    Pins the snapshot (the bests, taken before any import), the cadence (after
    generation exch_every's selection) and the import count."""
    base = configs.crs_line(2, n_cmp=5, ns=80, n_events=2, ap_half=1, np_=8, ng=3,
                            exch_every=3, polish_steps=0, tau_max=0.28)
    prob = synth.line_problem(base.line, half_window=3, ap_half=1, cmps=[1, 2, 3],
                              t0_range=(30, 34))
    assert (prob.n_m0, prob.n_t0) == (3, 4)
    th_x, S_x, n_x = osearch.search(base.traces, base.mid, base.off, prob, base.de)
    de0 = configs.DEConfig(**{**vars(base.de), "exch_every": 0})
    th_0, S_0, n_0 = osearch.search(base.traces, base.mid, base.off, prob, de0)
    n_imports = 2 * (3 * 3 + 4 * 2)
    assert n_x - n_0 == n_imports
    for d in range(prob.n_dom):
        nb = ex.neighbours(d, prob.n_m0, prob.n_t0)
        s_imp = semblance_many(base.traces, base.mid, base.off, prob,
                               th_0[nb][None].astype(f32), domains=[d])[0].astype(f32)
        assert S_x[d] == max(f32(S_0[d]), *s_imp), d


def test_polish_ascends_by_the_scaled_gradient():
    """One polish step from a point below the peak moves by
    lr (hi - lo)^2 dS/dtheta, the gradient taken here by central differences
    of the FP64 semblance (independent of the adjoint), and raises S; five
    steps get strictly closer to the generating velocity."""
    wl = configs.cmp_search(0)
    x = wl.traces.astype(np.float64)
    ev = wl.line.events[0]
    t0 = int(round(ev[1] / wl.dt)) * wl.dt
    C = ev[4]
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    dm, h = np.zeros(48), wl.off.astype(float)
    start = np.array([C * 1.02])
    S0 = semblance(x, wl.dt, dm, h, t0, 0, start, 5)
    eps = 1e-4 * C
    g_fd = (semblance(x, wl.dt, dm, h, t0, 0, start + eps, 5) -
            semblance(x, wl.dt, dm, h, t0, 0, start - eps, 5)) / (2 * eps)
    th1, S1, n1 = osearch.polish_point(x, wl.dt, dm, h, t0, 0, 5, start, lo, hi, 1,
                                       wl.de.polish_lr)
    assert n1 == 2 and S1 > S0
    step = wl.de.polish_lr * (hi - lo) ** 2 * g_fd
    assert th1[0] - start[0] == pytest.approx(step[0], rel=1e-3)
    th5, S5, _ = osearch.polish_point(x, wl.dt, dm, h, t0, 0, 5, start, lo, hi, 5,
                                      wl.de.polish_lr)
    assert S5 > S0 and abs(th5[0] - C) < abs(start[0] - C)


def test_polish_keeps_the_best_iterate():
    """A step size far too large throws every later iterate to the bounds,
    where the coherence is lower: the polish returns the starting point and
    its semblance (it never lowers S)."""
    wl = configs.cmp_search(0)
    x = wl.traces.astype(np.float64)
    ev = wl.line.events[0]
    t0 = int(round(ev[1] / wl.dt)) * wl.dt
    C = ev[4]
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    dm, h = np.zeros(48), wl.off.astype(float)
    start = np.array([C * 1.02])
    S0 = semblance(x, wl.dt, dm, h, t0, 0, start, 5)
    lr = wl.de.polish_lr * 1e6
    eps = 1e-4 * C
    g_fd = (semblance(x, wl.dt, dm, h, t0, 0, start + eps, 5) -
            semblance(x, wl.dt, dm, h, t0, 0, start - eps, 5)) / (2 * eps)
    th1 = np.clip(start + lr * (hi - lo) ** 2 * g_fd, lo, hi)
    assert th1[0] in (lo[0], hi[0])
    assert semblance(x, wl.dt, dm, h, t0, 0, th1, 5) < S0  # the first step overshoots
    th, S, n = osearch.polish_point(x, wl.dt, dm, h, t0, 0, 5, start, lo, hi, 3, lr)
    assert n == 4 and S == S0 and np.array_equal(th, start)
