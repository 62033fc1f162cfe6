"""JADE control-parameter adaptation with an archive (TEST INFRASTRUCTURE).

Sec. 2.1.4: the search's control parameters are those of the cited JADE
(Zhang & Sanderson, IEEE TEC 2009), which adapts F and CR through a memory of
the values that produced successful children and keeps an archive of the
parents those children replaced. With the paper's p = 1 (Sec. 2.1.2-2.1.3)
one JADE generation of one domain is, in JADE's order:

1. For every member i draw CR_i ~ Normal(mu_CR, 0.1) clipped to [0, 1] and
   F_i ~ Cauchy(mu_F, 0.1), drawn again while F_i <= 0 and set to 1 when
   F_i > 1.
2. Mutant v = x_i + F_i (x_best - x_i) + F_i (x_r1 - x~_r2): r1 a member other
   than i, x~_r2 a member or an archived parent other than i and r1
   (current-to-pbest/1 with archive, p = 1); binomial crossover with CR_i and
   j_rand; the bound repair of ``oracle.de``.
3. Selection as in ``oracle.de`` (the child replaces its parent when its
   semblance is greater or equal). A child that is strictly better is a
   success: its parent enters the archive and (CR_i, F_i) enter S_CR, S_F.
   The archive holds at most NP parents: a parent arriving when it is full
   replaces a uniformly chosen entry.
4. If there were successes: mu_CR <- (1 - c) mu_CR + c mean(S_CR) and
   mu_F <- (1 - c) mu_F + c sum(S_F^2) / sum(S_F) (the Lehmer mean), c = 0.1.

Readings where neither the paper nor JADE fixes a detail:
* Initial mu_F, mu_CR: the configured F and CR (JADE's 0.5, 0.5 when so set).
* Success is strict improvement (JADE keeps the parent on ties; the selection
  here takes the child on ties, which then is not a success).
* The archive's random removal is done one arrival at a time: while it is
  full, an arriving parent overwrites entry floor(w NP / 2^32).
* A generation without successes leaves mu unchanged.
* Arithmetic: IEEE float32, one rounding per operation, in the order written
  in the code below (sums over successes in member order).
* Random numbers come from Philox4x32-10 (``oracle.philox``) keyed by the seed
  and domain, with the counter's generation field carrying a stream tag:
  normal draws 0x80000000 | g, Cauchy draws 0xC0000000 | g (g the generation
  whose trial is being built), archive draws 0x40000000 | g (g the
  generation of the trial being selected). Words are taken in pairs
  (v1, v2), each word mapped to the odd multiple of 2^-24 in (-1, 1)
  v = (2 (x >> 8) + 1 - 2^24) 2^-24, and the pair accepted when
  s = v1^2 + v2^2 < 1 (a uniform point of the unit disc): the normal variate
  is v1 sqrt(-2 ln s / s) (Marsaglia's polar method), the Cauchy variate is
  v1 / v2 (the cotangent of a uniform angle). At most 16 pairs are tried for
  a normal draw (then z = 0) and 32 for F (then F_i = mu_F).
* ln s is computed in float32 from s = m 2^e, m in [1/sqrt 2, sqrt 2), as
  e ln 2 + 2 atanh(r), r = (m - 1)/(m + 1), with the atanh series
  r (1 + r^2/3 + ... + r^12/13) (Abramowitz & Stegun 4.1.27-4.6.22 form),
  so that only correctly rounded operations are involved.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import de as de_mod
from .philox import words

f32 = np.float32
C_ADAPT = f32(0.1)        # JADE's c
SIGMA = f32(0.1)          # spread of both CR (normal) and F (Cauchy)
NORMAL_TRIES, CAUCHY_TRIES = 16, 32
TAG_NORMAL, TAG_CAUCHY, TAG_ARCHIVE = 0x80000000, 0xC0000000, 0x40000000
LN2 = f32(0.6931471805599453)
INV_ODD = [f32(f32(1.0) / f32(2 * k + 1)) for k in range(7)]
RSQRT2 = f32(0.70710677)


def ln_f32(s) -> np.float32:
    """Natural log of a positive float32 by the atanh series, float32 ops."""
    s = f32(s)
    m, e = math.frexp(float(s))       # exact: s = m 2^e, m in [0.5, 1)
    m = f32(m)
    if m < RSQRT2:
        m = f32(m * f32(2.0))
        e -= 1
    r = f32(f32(m - f32(1.0)) / f32(m + f32(1.0)))
    r2 = f32(r * r)
    p = INV_ODD[6]
    for k in range(5, -1, -1):
        p = f32(f32(p * r2) + INV_ODD[k])
    t = f32(f32(f32(2.0) * r) * p)
    return f32(f32(f32(e) * LN2) + t)


def signed_unit(x: int) -> np.float32:
    """Odd multiple of 2^-24 in (-1, 1) from the top 24 bits of a word."""
    return f32((2 * (int(x) >> 8) + 1 - (1 << 24)) * 2.0 ** -24)


def _pairs(seed, d, tag_gen, i, n_pairs):
    w = words(seed, d, tag_gen, i, 2 * n_pairs)
    for k in range(n_pairs):
        v1, v2 = signed_unit(w[2 * k]), signed_unit(w[2 * k + 1])
        s = f32(f32(v1 * v1) + f32(v2 * v2))
        yield v1, v2, s


def normal_draw(seed, d, g, i) -> np.float32:
    """Standard normal variate (polar method), 0 if no pair is accepted."""
    for v1, v2, s in _pairs(seed, d, TAG_NORMAL | g, i, NORMAL_TRIES):
        if s < f32(1.0):
            q = f32(f32(f32(-2.0) * ln_f32(s)) / s)
            return f32(v1 * f32(np.sqrt(q)))
    return f32(0.0)


def draw_cr(seed, d, g, i, mu_cr) -> np.float32:
    z = normal_draw(seed, d, g, i)
    cr = f32(f32(mu_cr) + f32(SIGMA * z))
    return f32(min(max(cr, f32(0.0)), f32(1.0)))


def draw_f(seed, d, g, i, mu_f) -> np.float32:
    """Cauchy(mu_F, 0.1), redrawn while <= 0, truncated to 1."""
    for v1, v2, s in _pairs(seed, d, TAG_CAUCHY | g, i, CAUCHY_TRIES):
        if s < f32(1.0):
            F = f32(f32(mu_f) + f32(SIGMA * f32(v1 / v2)))
            if F > f32(0.0):
                return f32(min(F, f32(1.0)))
    return f32(mu_f)


def cr_threshold_f32(cr) -> int:
    """floor(CR_i 2^24) for a float32 CR_i in [0, 1] (the product is exact)."""
    return int(math.floor(float(f32(cr)) * 16777216.0))


@dataclass
class State:
    """Adaptation state of one domain."""
    mu_cr: np.float32
    mu_f: np.float32
    archive: np.ndarray      # [NP, D] float32, first n_arc rows valid
    n_arc: int
    F: np.ndarray            # [NP] F_i of the current trial
    CR: np.ndarray           # [NP] CR_i of the current trial


def new_state(NP, D, F0, CR0) -> State:
    return State(f32(CR0), f32(F0), np.zeros((NP, D), f32), 0, np.zeros(NP, f32),
                 np.zeros(NP, f32))


def mutation_draws(seed, d, g, i, NP, n_arc, D):
    """(r1, r2, j_rand, crossover words): r2 indexes members then archive."""
    w = words(seed, d, g, i, 3 + D)
    r1 = de_mod.index_below(w[0], NP - 1)
    if r1 >= i:
        r1 += 1
    r2 = de_mod.index_below(w[1], NP + n_arc - 2)
    a, b = min(i, r1), max(i, r1)
    if r2 >= a:
        r2 += 1
    if r2 >= b:
        r2 += 1
    jr = de_mod.index_below(w[2], D)
    return r1, r2, jr, w[3:3 + D]


def trial_population(st: State, seed, d, g, pop, fit, lo, hi):
    """Steps 1-2 for every member: draws (stored in st.F, st.CR) and the
    trial population of generation g; returns (trial, best index)."""
    NP, D = pop.shape
    b = de_mod.best_index(fit)
    trial = np.empty_like(pop)
    for i in range(NP):
        st.CR[i] = draw_cr(seed, d, g, i, st.mu_cr)
        st.F[i] = draw_f(seed, d, g, i, st.mu_f)
        thr = cr_threshold_f32(st.CR[i])
        F = st.F[i]
        r1, r2, jr, cw = mutation_draws(seed, d, g, i, NP, st.n_arc, D)
        x2 = pop[r2] if r2 < NP else st.archive[r2 - NP]
        xi, xb, x1 = pop[i], pop[b], pop[r1]
        for k in range(D):
            if (int(cw[k]) >> 8) < thr or k == jr:
                v = f32(f32(xi[k] + f32(F * f32(xb[k] - xi[k]))) + f32(F * f32(x1[k] - x2[k])))
            else:
                v = f32(xi[k])
            if v < f32(lo[k]):
                v = f32(f32(f32(lo[k]) + xi[k]) * f32(0.5))
            elif v > f32(hi[k]):
                v = f32(f32(f32(hi[k]) + xi[k]) * f32(0.5))
            trial[i, k] = v
    return trial, b


def select_adapt(st: State, seed, d, g_trial, pop, fit, trial, tfit):
    """Steps 3-4: selection of the trial of generation g_trial with the
    archive and memory updates; returns the new (pop, fit)."""
    NP = pop.shape[0]
    pop, fit = pop.copy(), fit.copy()
    s_cr = s_f = s_f2 = f32(0.0)
    n_succ = 0
    for i in range(NP):
        new, old = de_mod.rank_key(tfit[i]), de_mod.rank_key(fit[i])
        if new > old:
            if st.n_arc < NP:
                slot = st.n_arc
                st.n_arc += 1
            else:
                w = words(seed, d, TAG_ARCHIVE | g_trial, i, 1)[0]
                slot = de_mod.index_below(w, NP)
            st.archive[slot] = pop[i]
            s_cr = f32(s_cr + st.CR[i])
            s_f = f32(s_f + st.F[i])
            s_f2 = f32(s_f2 + f32(st.F[i] * st.F[i]))
            n_succ += 1
        if new >= old:
            pop[i], fit[i] = trial[i], tfit[i]
    if n_succ:
        omc = f32(f32(1.0) - C_ADAPT)
        mean_cr = f32(s_cr / f32(n_succ))
        lehmer = f32(s_f2 / s_f)
        st.mu_cr = f32(f32(omc * st.mu_cr) + f32(C_ADAPT * mean_cr))
        st.mu_f = f32(f32(omc * st.mu_f) + f32(C_ADAPT * lehmer))
    return pop, fit
