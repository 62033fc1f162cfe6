"""One generation of differential evolution per domain (TEST INFRASTRUCTURE).

Follows the JADE steps of Sec. 2.1 with the paper's p = 1 (so
DE/current-to-best/1, Sec. 2.1.3) and the control parameters F and CR held
fixed (the adaptive memory of Sec. 2.1.4 is not part of this search):

* Initialise (Sec. 2.1.1): theta_d = lo_d + u (hi_d - lo_d), u uniform.
* Best (Sec. 2.1.2, p = 1): argmax of the semblance, lowest index on ties,
  NaN ranked below every number.
* Mutation (Sec. 2.1.3): v = x_i + F (x_best - x_i) + F (x_r1 - x_r2),
  r1 != r2 != i uniform. (Sec. 2 also mentions Gaussian noise vectors; the
  JADE description of Sec. 2.1.3 is followed.)
* Binomial crossover with j_rand, then JADE's bound repair
  (v < lo -> (lo + x_i)/2, v > hi -> (hi + x_i)/2).
* Selection (Sec. 2.1.4): the child replaces its parent when its semblance
  is greater or equal.

Arithmetic is IEEE float32, one rounding per operation, in the order
written above (no fused multiply-add); the bound-repair branch and the
selection are decisions taken on these float32 values. Random numbers come
from Philox4x32-10 (``oracle.philox``): for (domain d, generation g,
individual i) the word stream is w0, w1, ...; at g = 0 word k initialises
dimension k; at g >= 1 w0 -> r1, w1 -> r2, w2 -> j_rand and w(3+k) is the
crossover word of dimension k. A word x maps to an index below n as
floor(x n / 2^32) (integer multiply-shift) and to a uniform in [0, 1) as
(x >> 8) 2^-24.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import words

f32 = np.float32


def index_below(x: int, n: int) -> int:
    """floor(x * n / 2^32) for a 32-bit word x: uniform-ish index in [0, n)."""
    return (int(x) * int(n)) >> 32


def unit_float(x: int) -> np.float32:
    """(x >> 8) * 2^-24, exactly representable in float32, in [0, 1)."""
    return f32((int(x) >> 8) * 2.0 ** -24)


def cr_threshold(CR: float) -> int:
    """Crossover threshold on 24-bit draws: floor(float32(CR) * 2^24)."""
    return int(math.floor(float(f32(CR)) * 16777216.0))


def rank_key(v) -> float:
    """Fitness with NaN ranked below every number."""
    v = float(v)
    return -math.inf if math.isnan(v) else v


def best_index(fit) -> int:
    """argmax of the fitness, lowest index on ties, NaN lowest."""
    best, bk = 0, rank_key(fit[0])
    for i in range(1, len(fit)):
        k = rank_key(fit[i])
        if k > bk:
            best, bk = i, k
    return best


def init_individual(seed, d, i, lo, hi, gen=0):
    """Initial individual i of domain d: lo + u (hi - lo) in float32, from the
    words of counter generation ``gen`` (0 for the search's generation 0)."""
    D = len(lo)
    w = words(seed, d, gen, i, D)
    out = np.empty(D, f32)
    for k in range(D):
        out[k] = f32(lo[k]) + unit_float(w[k]) * (f32(hi[k]) - f32(lo[k]))
    return out


def mutation_draws(seed, d, g, i, NP, D):
    """(r1, r2, j_rand, crossover words) for individual i at generation g."""
    w = words(seed, d, g, i, 3 + D)
    r1 = index_below(w[0], NP - 1)
    if r1 >= i:
        r1 += 1
    r2 = index_below(w[1], NP - 2)
    a, b = min(i, r1), max(i, r1)
    if r2 >= a:
        r2 += 1
    if r2 >= b:
        r2 += 1
    jr = index_below(w[2], D)
    return r1, r2, jr, w[3:3 + D]


def trial_individual(seed, d, g, i, pop, best, F, CR, lo, hi):
    """Mutant + binomial crossover + bound repair for individual i."""
    NP, D = pop.shape
    r1, r2, jr, cw = mutation_draws(seed, d, g, i, NP, D)
    F = f32(F)
    thr = cr_threshold(CR)
    xi, xb, x1, x2 = pop[i], pop[best], pop[r1], pop[r2]
    out = np.empty(D, f32)
    for k in range(D):
        if (int(cw[k]) >> 8) < thr or k == jr:
            v = f32(f32(xi[k] + f32(F * f32(xb[k] - xi[k]))) + f32(F * f32(x1[k] - x2[k])))
        else:
            v = f32(xi[k])
        if v < f32(lo[k]):
            v = f32(f32(f32(lo[k]) + xi[k]) * f32(0.5))
        elif v > f32(hi[k]):
            v = f32(f32(f32(hi[k]) + xi[k]) * f32(0.5))
        out[k] = v
    return out


def select(pop, fit, trial, trial_fit):
    """Greedy selection: child replaces parent when S_child >= S_parent."""
    pop, fit = pop.copy(), fit.copy()
    for i in range(pop.shape[0]):
        if rank_key(trial_fit[i]) >= rank_key(fit[i]):
            pop[i] = trial[i]
            fit[i] = trial_fit[i]
    return pop, fit


def init_population(seed, d, NP, lo, hi):
    return np.stack([init_individual(seed, d, i, lo, hi) for i in range(NP)])


def mutate_population(seed, d, g, pop, fit, F, CR, lo, hi):
    """Trial population of generation g (>= 1) and the best index used."""
    b = best_index(fit)
    trial = np.stack([trial_individual(seed, d, g, i, pop, b, F, CR, lo, hi)
                      for i in range(pop.shape[0])])
    return trial, b


def de_step(gen, pop, fit, trial, trial_fit, seed, F, CR, lo, hi, *, domains=None,
            mutate=True):
    """One DE step over many domains, mirroring the library entry point.

    gen == 0: returns the initial population (pop/fit ignored).
    gen >= 1: if ``trial`` is given, first selects it into (pop, fit); then,
    if ``mutate``, builds the trial of generation ``gen``. Returns
    (pop, fit, next_trial or None, best_idx) as new float32 arrays.
    """
    lo = np.asarray(lo, f32)
    hi = np.asarray(hi, f32)
    n_dom = pop.shape[0]
    doms = range(n_dom) if domains is None else domains
    if gen == 0:
        NP = pop.shape[1]
        newpop = np.stack([init_population(seed, d, NP, lo, hi) for d in doms])
        return newpop, None, None, None
    pop = np.array(pop, f32)
    fit = np.array(fit, f32)
    nxt = np.empty_like(pop) if mutate else None
    best = np.empty(n_dom, np.int32)
    for r, d in enumerate(doms):
        if trial is not None:
            pop[r], fit[r] = select(pop[r], fit[r], trial[r], trial_fit[r])
        if mutate:
            nxt[r], best[r] = mutate_population(seed, d, gen, pop[r], fit[r], F, CR, lo, hi)
        else:
            best[r] = best_index(fit[r])
    return pop, fit, nxt, best
