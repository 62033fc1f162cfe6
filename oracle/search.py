"""The whole traveltime-parameter search (TEST INFRASTRUCTURE).

Per domain (zero-offset sample) the JADE loop of Sec. 2.1 / Fig. 3 with
p = 1, with fixed F, CR (``oracle.de``) or, when ``cfg.adapt`` is set, with
JADE's adaptation of F and CR and its archive (``oracle.jade``), driven over
all domains at once with the neighbour exchange of Sec. 3.3
(``oracle.exchange``):

    gen 0:          init population, evaluate it
    gen g = 1..NG:  best -> mutate/crossover -> evaluate trial -> select
                    if exch_every > 0 and g % exch_every == 0:
                        snapshot bests, import neighbours' bests into the
                        worst slots, evaluate them at the receiving domain
    result:         best member (argmax, lowest index on ties)
    polish:         polish_steps projected gradient-ascent steps on S from
                    the DE winner (an addition to the paper's method):
                    theta <- clip(theta + lr (hi - lo)^2 * dS/dtheta, lo, hi),
                    i.e. plain ascent in coordinates scaled to the bounds;
                    S is evaluated at every iterate and the best iterate
                    (first on ties) is kept, so polishing never lowers S.

Semblance is FP64 (``oracle.semblance``) and stored as float32 fitness, the
precision the DE decisions are taken in; the polish runs in FP64.
Returns (best_theta [n_dom, D] float64, best_S [n_dom], n_evals).
"""
from __future__ import annotations

import numpy as np

from . import de as de_mod
from . import exchange as ex
from . import jade
from .semblance import semblance_many, domain_data, semblance, semblance_grad


def _eval(traces, mid, off, prob, theta):
    return semblance_many(traces, mid, off, prob, theta).astype(np.float32)


def polish_point(x, dt, dm, h, t0, op, w, theta0, lo, hi, steps, lr):
    """Projected gradient ascent from theta0; returns (theta, S, n_calls)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    scale = lr * (hi - lo) ** 2
    th = np.asarray(theta0, np.float64).copy()
    best_th, best_S = th.copy(), None
    for _ in range(steps):
        S, g = semblance_grad(x, dt, dm, h, t0, op, th, w)
        if best_S is None or S > best_S:
            best_th, best_S = th.copy(), S
        th = np.clip(th + scale * g, lo, hi)
    S = semblance(x, dt, dm, h, t0, op, th, w)
    if best_S is None or S > best_S:
        best_th, best_S = th.copy(), S
    return best_th, best_S, steps + 1


def search(traces, mid, off, prob, cfg, *, history=None, jade_states=None, dom_base=0,
           halo=None):
    """Run the search over every domain of ``prob`` with settings ``cfg``
    (attributes np, ng, F, CR, seed, lo, hi, exch_every, polish_steps,
    polish_lr and optionally adapt). ``history``, if a list, receives the
    mean best S per gen; ``jade_states``, if a list, the final adaptation
    state of every domain.

    One slab of a longer line: ``dom_base`` is the global index of the
    grid's first domain (it keys the random numbers, so a slab draws what
    the whole-line search draws for the same domains), and ``halo``, if
    given, is called at every exchange as halo(g, first_row, last_row) with
    the snapshot bests of the slab's first and last m0 rows [n_t0, D]; it
    returns the bests of the neighbouring slabs' adjacent rows (prev_row,
    next_row), None where the slab is at a line end."""
    lo = np.asarray(cfg.lo, np.float32)
    hi = np.asarray(cfg.hi, np.float32)
    n_dom, NP, D = prob.n_dom, cfg.np, len(cfg.lo)
    gdoms = range(dom_base, dom_base + n_dom)
    pop = np.zeros((n_dom, NP, D), np.float32)
    pop, _, _, _ = de_mod.de_step(0, pop, None, None, None, cfg.seed, cfg.F, cfg.CR, lo, hi,
                                  domains=gdoms)
    fit = _eval(traces, mid, off, prob, pop)
    n_evals = n_dom * NP
    grid = cfg.exch_every > 0 and prob.n_m0 * prob.n_t0 == n_dom and n_dom > 0
    adapt = bool(getattr(cfg, "adapt", 0))
    states = [jade.new_state(NP, D, cfg.F, cfg.CR) for _ in range(n_dom)] if adapt else None
    for g in range(1, cfg.ng + 1):
        if adapt:
            trial = np.empty_like(pop)
            for d in range(n_dom):
                trial[d], _ = jade.trial_population(states[d], cfg.seed, dom_base + d, g,
                                                    pop[d], fit[d], lo, hi)
        else:
            pop, fit, trial, _ = de_mod.de_step(g, pop, fit, None, None, cfg.seed, cfg.F,
                                                cfg.CR, lo, hi, domains=gdoms)
        tfit = _eval(traces, mid, off, prob, trial)
        n_evals += n_dom * NP
        for d in range(n_dom):
            if adapt:
                pop[d], fit[d] = jade.select_adapt(states[d], cfg.seed, dom_base + d, g, pop[d],
                                                   fit[d], trial[d], tfit[d])
            else:
                pop[d], fit[d] = de_mod.select(pop[d], fit[d], trial[d], tfit[d])
        if grid and g % cfg.exch_every == 0:
            snap = ex.best_snapshot(pop, fit)
            prev_row = next_row = None
            if halo is not None:
                prev_row, next_row = halo(g, snap[:prob.n_t0].copy(), snap[-prob.n_t0:].copy())
            imports, slots = ex.exchange_plan(prob.n_m0, prob.n_t0, pop, fit, snap,
                                              prev_row, next_row)
            ifit = _eval(traces, mid, off, prob, imports)
            ifit[slots < 0] = 0.0
            n_evals += int(np.sum(slots >= 0))
            pop, fit = ex.apply_exchange(pop, fit, imports, slots, ifit)
        if history is not None:
            history.append(float(np.mean([fit[d, de_mod.best_index(fit[d])]
                                          for d in range(n_dom)])))
    bidx = np.array([de_mod.best_index(fit[d]) for d in range(n_dom)])
    best_theta = pop[np.arange(n_dom), bidx].astype(np.float64)
    best_S = fit[np.arange(n_dom), bidx].astype(np.float64)
    if cfg.polish_steps > 0:
        for d in range(n_dom):
            x, dt, dm, h, t0 = domain_data(traces, mid, off, prob, d)
            best_theta[d], best_S[d], n = polish_point(
                x, dt, dm, h, t0, prob.op, prob.half_window, best_theta[d], lo, hi,
                cfg.polish_steps, cfg.polish_lr)
            n_evals += n
    if adapt and jade_states is not None:
        jade_states.extend(states)
    return best_theta, best_S, n_evals
