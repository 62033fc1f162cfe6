"""Pins of the oracle's random numbers and DE step.

Philox4x32-10 against its published known-answer vectors; index and
crossover draws against their defining properties (ranges, exclusions,
uniformity); mutation, repair and selection against closed forms.
"""
import math
import os

import numpy as np
import pytest

from oracle import de, philox

f32 = np.float32


def test_philox_known_answers(golden_dir):
    n = 0
    for line in open(os.path.join(golden_dir, "philox4x32_10_kat.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        v = [int(t, 16) for t in line.split()]
        assert philox.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])
        n += 1
    assert n == 3


def test_words_stream_layout():
    seed = 0x0123456789ABCDEF
    w = philox.words(seed, 7, 3, 5, 9)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    assert w[:4] == list(philox.philox4x32_10((5, 3, 7, 0), key))
    assert w[4:8] == list(philox.philox4x32_10((5, 3, 7, 1), key))
    assert w[8] == philox.philox4x32_10((5, 3, 7, 2), key)[0]


def test_index_below_bounds_and_monotone():
    for n in (1, 2, 3, 5, 31, 63, 95, 1000):
        assert de.index_below(0, n) == 0
        assert de.index_below(0xFFFFFFFF, n) == n - 1
        # boundaries: the first word mapping to k is ceil(k 2^32 / n)
        for k in range(1, min(n, 20)):
            b = -(-(k << 32) // n)
            assert de.index_below(b, n) == k
            assert de.index_below(b - 1, n) == k - 1


def test_unit_float_range_exact():
    assert de.unit_float(0) == 0.0
    assert de.unit_float(0xFFFFFFFF) == f32(1.0 - 2.0 ** -24)
    assert de.unit_float(0xFFFFFFFF) < 1.0
    assert de.unit_float(1 << 31) == 0.5


def test_cr_threshold():
    assert de.cr_threshold(0.0) == 0
    assert de.cr_threshold(1.0) == 1 << 24
    assert de.cr_threshold(0.5) == 1 << 23
    # float32(0.9) = 0x3F666666: significand 0xE66666 scaled by 2^-24 exactly
    assert de.cr_threshold(0.9) == 0xE66666 == 15099494


def test_mutation_draws_exclusions_and_uniformity():
    NP, D = 8, 3
    counts1 = np.zeros(NP, int)
    counts2 = np.zeros(NP, int)
    countsj = np.zeros(D, int)
    for d in range(40):
        for g in range(1, 26):
            for i in range(NP):
                r1, r2, jr, cw = de.mutation_draws(11, d, g, i, NP, D)
                assert 0 <= r1 < NP and 0 <= r2 < NP and 0 <= jr < D
                assert r1 != i and r2 != i and r2 != r1
                assert len(cw) == D
                if i == 0:
                    counts1[r1] += 1
                    counts2[r2] += 1
                countsj[jr] += 1
    # i = 0: r1 uniform over 1..7, r2 uniform over the 6 others given r1
    n = counts1.sum()
    assert counts1[0] == 0 and counts2[0] == 0
    exp = n / (NP - 1)
    chi1 = np.sum((counts1[1:] - exp) ** 2 / exp)
    chi2 = np.sum((counts2[1:] - exp) ** 2 / exp)
    assert chi1 < 24.3 and chi2 < 24.3  # chi^2(6) at p = 0.9995
    expj = countsj.sum() / D
    assert np.sum((countsj - expj) ** 2 / expj) < 15.2  # chi^2(2) at p = 0.9995


def test_draws_depend_on_every_key_field():
    base = de.mutation_draws(1, 2, 3, 4, 64, 3)
    for args in [(2, 2, 3, 4), (1, 3, 3, 4), (1, 2, 4, 4), (1, 2, 3, 5)]:
        other = de.mutation_draws(*args, 64, 3)
        assert other != base


def _pop(NP, D, rng):
    return rng.uniform(-1, 1, (NP, D)).astype(f32)


def test_crossover_cr_zero_takes_only_jrand():
    rng = np.random.default_rng(0)
    NP, D = 10, 3
    lo, hi = np.full(D, -100, f32), np.full(D, 100, f32)
    pop = _pop(NP, D, rng)
    for i in range(NP):
        r1, r2, jr, _ = de.mutation_draws(5, 0, 1, i, NP, D)
        t = de.trial_individual(5, 0, 1, i, pop, 0, 0.5, 0.0, lo, hi)
        for k in range(D):
            if k == jr:
                v = pop[i, k] + 0.5 * (pop[0, k] - pop[i, k]) + 0.5 * (pop[r1, k] - pop[r2, k])
                assert t[k] == pytest.approx(v, rel=1e-6, abs=1e-7)
            else:
                assert t[k] == pop[i, k]


def test_crossover_cr_one_takes_all_and_f_one_closed_form():
    rng = np.random.default_rng(1)
    NP, D = 12, 3
    lo, hi = np.full(D, -100, f32), np.full(D, 100, f32)
    pop = _pop(NP, D, rng)
    b = 4
    for i in range(NP):
        r1, r2, jr, _ = de.mutation_draws(9, 2, 7, i, NP, D)
        t = de.trial_individual(9, 2, 7, i, pop, b, 1.0, 1.0, lo, hi)
        # F = 1: v = x_i + (x_b - x_i) + (x_r1 - x_r2) = x_b + x_r1 - x_r2
        np.testing.assert_allclose(t, pop[b] + pop[r1] - pop[r2], rtol=1e-6, atol=1e-6)


def test_crossover_rate_matches_cr():
    rng = np.random.default_rng(2)
    NP, D = 16, 3
    lo, hi = np.full(D, -100, f32), np.full(D, 100, f32)
    pop = _pop(NP, D, rng)
    taken = total = 0
    for g in range(1, 200):
        for i in range(NP):
            _, _, jr, _ = de.mutation_draws(3, 1, g, i, NP, D)
            t = de.trial_individual(3, 1, g, i, pop, 0, 0.5, 0.3, lo, hi)
            for k in range(D):
                if k != jr:
                    total += 1
                    taken += int(t[k] != pop[i, k])
    assert taken / total == pytest.approx(0.3, abs=0.03)


def test_identical_population_is_fixed_point():
    NP, D = 6, 3
    pop = np.tile(np.array([0.1, -0.2, 0.3], f32), (NP, 1))
    lo, hi = np.full(D, -1, f32), np.full(D, 1, f32)
    for i in range(NP):
        np.testing.assert_array_equal(de.trial_individual(1, 0, 1, i, pop, 2, 0.5, 0.9, lo, hi),
                                      pop[i])


def test_bound_repair_closed_form():
    NP, D = 5, 1
    lo, hi = np.array([0.0], f32), np.array([1.0], f32)
    # best at hi, the difference pushes far beyond: repaired to (hi + x_i)/2
    for i in range(1, NP):
        pop = np.array([[1.0], [0.2], [0.4], [0.6], [0.8]], f32)
        r1, r2, jr, _ = de.mutation_draws(4, 0, 1, i, NP, D)
        v = pop[i, 0] + 1.0 * (pop[0, 0] - pop[i, 0]) + 1.0 * (pop[r1, 0] - pop[r2, 0])
        t = de.trial_individual(4, 0, 1, i, pop, 0, 1.0, 1.0, lo, hi)[0]
        if v > 1.0:
            assert t == f32((1.0 + pop[i, 0]) / 2)
        elif v < 0.0:
            assert t == f32((0.0 + pop[i, 0]) / 2)
        else:
            assert t == pytest.approx(v, abs=1e-6)
    # a population at the lower edge with a negative push
    pop = np.array([[0.0], [0.0], [0.5], [0.0], [0.0]], f32)
    for i in (1, 3, 4):
        r1, r2, _, _ = de.mutation_draws(8, 0, 1, i, NP, D)
        t = de.trial_individual(8, 0, 1, i, pop, 0, 1.0, 1.0, lo, hi)[0]
        assert 0.0 <= t <= 1.0
        if pop[r1, 0] - pop[r2, 0] < 0:
            assert t == 0.0


def test_selection_rule():
    pop = np.zeros((4, 2), f32)
    trial = np.ones((4, 2), f32)
    fit = np.array([0.5, 0.5, np.nan, 0.2], f32)
    tfit = np.array([0.4, 0.5, 0.1, np.nan], f32)
    p, f = de.select(pop, fit, trial, tfit)
    np.testing.assert_array_equal(p[:, 0], [0, 1, 1, 0])  # lower, tie wins, beats NaN, NaN loses
    assert f[1] == 0.5 and f[2] == f32(0.1)


def test_best_index_ties_and_nan():
    assert de.best_index([0.1, 0.7, 0.7, 0.2]) == 1
    assert de.best_index([np.nan, 0.0, 0.0]) == 1
    assert de.best_index([np.nan, np.nan]) == 0
    assert de.best_index([-1.0, np.nan, -0.5]) == 2


def test_init_uniform_in_bounds():
    lo = np.array([-6e-4, -1.5e-7, 4.34e-8], f32)
    hi = np.array([6e-4, 1.5e-7, 5.1e-7], f32)
    pops = np.stack([de.init_population(0, d, 64, lo, hi) for d in range(50)])
    assert np.all(pops >= lo) and np.all(pops <= hi)
    z = (pops - lo) / (hi - lo)
    assert np.mean(z) == pytest.approx(0.5, abs=0.01)
    assert np.var(z) == pytest.approx(1 / 12, abs=0.005)
    # exact float32 formula on one draw: lo + u (hi - lo), u = (w >> 8) 2^-24
    w = philox.words(0, 3, 0, 5, 3)
    for k in range(3):
        u = f32((w[k] >> 8) * 2.0 ** -24)
        assert pops[3, 5, k] == f32(lo[k] + f32(u * f32(hi[k] - lo[k])))


def test_de_step_select_then_mutate_equals_parts():
    rng = np.random.default_rng(3)
    n_dom, NP, D = 3, 8, 3
    lo, hi = np.full(D, -1, f32), np.full(D, 1, f32)
    pop = rng.uniform(-1, 1, (n_dom, NP, D)).astype(f32)
    fit = rng.uniform(0, 1, (n_dom, NP)).astype(f32)
    tr = rng.uniform(-1, 1, (n_dom, NP, D)).astype(f32)
    tf = rng.uniform(0, 1, (n_dom, NP)).astype(f32)
    p1, f1, nxt, b = de.de_step(5, pop, fit, tr, tf, 42, 0.5, 0.9, lo, hi)
    p2, f2, _, _ = de.de_step(5, pop, fit, tr, tf, 42, 0.5, 0.9, lo, hi, mutate=False)
    np.testing.assert_array_equal(p1, p2)
    _, _, nxt2, b2 = de.de_step(5, p2, f2, None, None, 42, 0.5, 0.9, lo, hi)
    np.testing.assert_array_equal(nxt, nxt2)
    np.testing.assert_array_equal(b, b2)
    for d in range(n_dom):
        assert b[d] == int(np.argmax(f1[d]))
