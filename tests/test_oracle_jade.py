"""Pins of the JADE adaptation oracle (oracle.jade).

* ln_f32 against the library logarithm (error bound) and exact at powers of 2.
* The word-to-(-1, 1) map: extremes, symmetry, never 0.
* Normal draws pass a Kolmogorov-Smirnov test against N(0, 1), with the
  polar method's acceptance rate pi/4; the F draws follow the Cauchy
  distribution truncated as JADE prescribes; CR clipping mass matches the
  normal tail.
* The memory update on hand-computed values (arithmetic and Lehmer means).
* The archive: fills in member order, never exceeds NP, holds only replaced
  parents, full-archive replacements are uniform; ties are not successes.
* r2 ranges over members and archive, never i or r1, uniformly.
* Reduction: with an empty archive and the draws forced to constants, one
  generation equals the fixed-parameter DE of ``oracle.de`` bit for bit.
* End to end: the adaptive search recovers the generating velocities of the
  CMP gather within 1%, and the memory stays inside (0, 1].
"""
import math

import numpy as np
import pytest

from oracle import de, jade, search as osearch
from oracle.philox import words
import synth
from synth import configs

f32 = np.float32
scipy_stats = pytest.importorskip("scipy.stats")


def test_ln_f32_bound_and_exact_points():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(1e-7, 1, 5000), 2.0 ** -rng.uniform(0, 47, 5000)])
    for x in xs.astype(f32):
        ref = math.log(float(x))
        assert abs(float(jade.ln_f32(x)) - ref) <= 3e-7 * abs(ref) + 1e-7, x
    assert jade.ln_f32(f32(1.0)) == 0.0
    for e in range(1, 40):
        assert jade.ln_f32(f32(2.0 ** -e)) == f32(f32(-e) * jade.LN2)


def test_signed_unit_map():
    assert jade.signed_unit(0) == f32(-1 + 2 ** -24)
    assert jade.signed_unit(0xFFFFFFFF) == f32(1 - 2 ** -24)
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2 ** 32, 2000, dtype=np.uint64):
        v = jade.signed_unit(int(x))
        assert v != 0 and -1 < v < 1
        assert jade.signed_unit(0xFFFFFFFF - int(x)) == -v


def test_normal_draws_are_standard_normal():
    z = np.array([jade.normal_draw(5, d, g, i) for d in range(4) for g in (1, 9)
                  for i in range(2500)], np.float64)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3
    # acceptance of the first pair: pi/4
    acc = np.mean([next(jade._pairs(5, 0, jade.TAG_NORMAL | 1, i, 1))[2] < 1
                   for i in range(20000)])
    assert abs(acc - math.pi / 4) < 0.01


def test_f_draws_follow_truncated_cauchy():
    mu = f32(0.3)
    F = np.array([jade.draw_f(9, d, 2, i, mu) for d in range(3) for i in range(4000)])
    assert np.all((F > 0) & (F <= 1))
    c = scipy_stats.cauchy(loc=0.3, scale=0.1)
    pos = 1 - c.cdf(0)
    for x in (0.1, 0.25, 0.3, 0.45, 0.8):
        expect = (c.cdf(x) - c.cdf(0)) / pos
        assert abs(np.mean(F < x) - expect) < 4 * math.sqrt(expect * (1 - expect) / F.size) + 1e-3
    expect1 = (1 - c.cdf(1)) / pos
    assert abs(np.mean(F == 1) - expect1) < 4 * math.sqrt(expect1 * (1 - expect1) / F.size) + 1e-3


def test_cr_draws_clip_at_the_normal_tail():
    CR = np.array([jade.draw_cr(4, 0, 3, i, f32(0.95)) for i in range(20000)])
    assert np.all((CR >= 0) & (CR <= 1))
    tail = 1 - scipy_stats.norm.cdf(0.5)   # P(0.95 + 0.1 z > 1)
    assert abs(np.mean(CR == 1) - tail) < 0.015
    # and at the lower end: CR_i = 0 with the mass of the tail below 0
    CR0 = np.array([jade.draw_cr(4, 1, 3, i, f32(0.05)) for i in range(20000)])
    low = scipy_stats.norm.cdf(-0.5)        # P(0.05 + 0.1 z < 0)
    assert abs(np.mean(CR0 == 0) - low) < 0.015
    assert np.all((CR0 >= 0) & (CR0 <= 1))
    assert jade.cr_threshold_f32(f32(1.0)) == 1 << 24
    assert jade.cr_threshold_f32(f32(0.0)) == 0


def test_normal_draw_is_the_first_polar_variate():
    """Marsaglia's polar method on the first accepted pair (v1, v2) of the
    member's words gives two normals, v1 sqrt(-2 ln s / s) and
    v2 sqrt(-2 ln s / s); the draw is the first. Recomputed here in FP64 from
    the pair (the FP32 logarithm and square root agree to a few ulp)."""
    for i in range(300):
        for v1, v2, s in jade._pairs(7, 3, jade.TAG_NORMAL | 5, i, jade.NORMAL_TRIES):
            if s < 1:
                q = -2.0 * math.log(float(s)) / float(s)
                z1 = float(v1) * math.sqrt(q)
                break
        z = float(jade.normal_draw(7, 3, 5, i))
        assert abs(z - z1) <= 2e-6 * max(1.0, abs(z1)), (i, z, z1)


def test_memory_update_hand_values():
    """Two successes, F = (0.5, 1.0), CR = (0.2, 0.4), mu = (0.5, 0.5):
    Lehmer mean (0.25 + 1) / 1.5 = 5/6, mu_F = 0.9 * 0.5 + 0.1 * 5/6 = 8/15;
    mean CR 0.3, mu_CR = 0.45 + 0.03 = 0.48. Member 2 ties (no success)."""
    st = jade.new_state(4, 1, 0.5, 0.5)
    st.F[:] = [0.5, 1.0, 0.7, 0.9]
    st.CR[:] = [0.2, 0.4, 0.9, 0.1]
    pop = np.array([[1], [2], [3], [4]], f32)
    fit = np.array([0.1, 0.2, 0.3, 0.9], f32)
    trial = np.array([[5], [6], [7], [8]], f32)
    tfit = np.array([0.5, 0.6, 0.3, 0.2], f32)
    p2, f2 = jade.select_adapt(st, 1, 0, 1, pop, fit, trial, tfit)
    assert st.mu_f == pytest.approx(8 / 15, abs=1e-7)
    assert st.mu_cr == pytest.approx(0.48, abs=1e-7)
    np.testing.assert_array_equal(p2[:, 0], [5, 6, 7, 4])   # the tie takes the child
    assert st.n_arc == 2
    np.testing.assert_array_equal(st.archive[:2, 0], [1, 2])
    # no success: memory unchanged
    mu = (st.mu_f, st.mu_cr)
    jade.select_adapt(st, 1, 0, 2, p2, f2, p2, f2 - 1)
    assert (st.mu_f, st.mu_cr) == mu and st.n_arc == 2


def test_archive_fills_then_replaces_uniformly():
    NP = 8
    st = jade.new_state(NP, 1, 0.5, 0.5)
    st.F[:], st.CR[:] = 0.5, 0.5
    counts = np.zeros(NP, int)
    seen = set()
    for g in range(1, 400):
        pop = (np.arange(NP, dtype=f32) + 100 * g)[:, None]
        fit = np.zeros(NP, f32)
        before = st.archive.copy()
        jade.select_adapt(st, 3, 0, g, pop, fit, pop, np.ones(NP, f32))
        seen.update(pop[:, 0].tolist())
        assert st.n_arc == NP
        assert set(st.archive[:, 0].tolist()) <= seen
        if g > 1:
            counts += (st.archive[:, 0] != before[:, 0])
        if g == 1:
            np.testing.assert_array_equal(st.archive[:, 0], pop[:, 0])
    # each generation 8 arrivals land on uniform slots: every slot is hit often
    assert counts.min() > 0.5 * counts.mean()


def test_r2_over_members_and_archive():
    NP, n_arc, D = 6, 4, 3
    hits = np.zeros(NP + n_arc, int)
    for g in range(1, 3000):
        r1, r2, jr, cw = jade.mutation_draws(2, 5, g, 1, NP, n_arc, D)
        assert r1 != 1 and r2 not in (1, r1) and 0 <= r2 < NP + n_arc and 0 <= jr < D
        hits[r2] += 1
    assert hits[1] == 0
    # given r1, r2 is uniform over the NP + n_arc - 2 others: a member k != 1
    # is r2 with probability (1 - 1/(NP-1)) / (NP+n_arc-2), an archived parent
    # with 1 / (NP+n_arc-2)
    n = hits.sum()
    for k in range(NP + n_arc):
        if k == 1:
            continue
        p = (1 - 1 / (NP - 1)) / (NP + n_arc - 2) if k < NP else 1 / (NP + n_arc - 2)
        assert abs(hits[k] - n * p) < 5 * math.sqrt(n * p * (1 - p)), (k, hits[k], n * p)


def test_reduces_to_fixed_de_with_constant_draws(monkeypatch):
    rng = np.random.default_rng(4)
    NP, D = 12, 3
    lo, hi = np.array([-1, -2, 0], f32), np.array([1, 2, 3], f32)
    pop = (lo + rng.uniform(0, 1, (NP, D)) * (hi - lo)).astype(f32)
    fit = rng.uniform(0, 1, NP).astype(f32)
    monkeypatch.setattr(jade, "draw_cr", lambda *a: f32(0.7))
    monkeypatch.setattr(jade, "draw_f", lambda *a: f32(0.6))
    st = jade.new_state(NP, D, 0.6, 0.7)
    got, b = jade.trial_population(st, 77, 9, 5, pop, fit, lo, hi)
    ref, rb = de.mutate_population(77, 9, 5, pop, fit, 0.6, 0.7, lo, hi)
    assert b == rb
    np.testing.assert_array_equal(got, ref)


def test_adaptive_search_recovers_velocities():
    """The CMP gather's event-centred samples (plus their neighbours)."""
    wl = configs.cmp_search(0, ns=500, np_=16, ng=30)
    ev = [(int(round(e[1] / wl.dt)), e[4]) for e in wl.line.events]
    ev = [(it, C) for it, C in ev if 10 <= it < 490]
    it0 = sorted({it + k for it, _ in ev for k in (-1, 0, 1)})
    prob = synth.cmp_problem(wl.line, half_window=5, it0=it0)
    cfg = wl.de
    cfg.adapt, cfg.F, cfg.CR = 1, 0.5, 0.5
    states = []
    th, S, n = osearch.search(wl.traces, wl.mid, wl.off, prob, cfg, jade_states=states)
    assert n == prob.n_dom * 16 * 31
    assert all(0 < s.mu_f <= 1 and 0 <= s.mu_cr <= 1 and s.n_arc <= 16 for s in states)
    assert len({round(float(s.mu_f), 6) for s in states}) > 5   # the memory moved
    hits = sum(int(abs(th[it0.index(it), 0] - C) <= 0.01 * C) for it, C in ev)
    assert len(ev) >= 6 and hits >= len(ev) - 1, (hits, len(ev))
