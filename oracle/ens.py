"""Evolution by neighborhood similarity, sweep mode (TEST INFRASTRUCTURE).

The paper's ENS (Sec. 3.3 "Information propagation", Sec. 3.5 "The
performance-quality trade-off by an interpolation process", Sec. 3.6
"Evolution by neighborhood similarity") on a line of n_m0 output traces
(CMPs) x n_t0 samples, domains laid out m0-major (d = c n_t0 + t). The line
is cut into buckets of N_bucket consecutive traces (the interactive domain of
Sec. 4); buckets are independent and every bucket runs the same stages:

* stage 0, forward exploration (Sec. 3.6, first stage): traces left to right;
  at each trace the samples t = 0, N_skip+1, 2(N_skip+1), ... are estimated,
  each with NP_f individuals, one of which (from the bucket's second trace
  on) is the best of sample t on the previous trace, evolved for NG_f
  generations;
* then N_cycle backward-and-forward cycles (Sec. 3.6, second and third
  stages): the backward stage sweeps right to left estimating t = init_b +
  k (N_skip+1) (init_b = 0 if N_skip = 0, else 1), the forward stage sweeps
  left to right estimating t = N_skip + k (N_skip+1) (init 0, 1, 2 for
  N_skip = 0, 1, 2). Each estimated sample starts from NP_bf individuals: the
  bests of samples t-1 and t+1 on the same trace, the best of sample t on the
  previous trace of the sweep (absent on the sweep's first trace), and its
  own best (Sec. 3.3, the four seeds), the remaining members random; it is
  evolved for NG_bf generations;
* after the estimated samples of a trace, every other sample of that trace is
  interpolated linearly in t between the bests of the nearest estimated
  samples (Sec. 3.5; beyond the first / last estimated sample the nearest one
  is copied), its semblance is computed, and it replaces the sample's best
  when higher (in stage 0 it is the first value).

Readings taken where the paper is silent:
* The estimated samples of one trace are processed in parallel (Sec. 5,
  "done in parallel in the GPU"), so their seeds from samples t-1 and t+1 are
  the bests as they stood before the step; the previous trace's best is the
  one this stage has just produced.
* Seeds fill the first population slots in the order (t-1, t+1, previous
  trace, own best), absent ones skipped; the other slots are random.
* Random numbers: the DE draws of ``oracle.de`` with the counter generation
  set to (stage + 1) * 65536 + g for generation g (g = 0: the initial
  population's random members, keyed by their slot).
* Interpolation weights in float32: w = (t - ta) / (tb - ta) correctly
  rounded, theta = theta_a + w (theta_b - theta_a), one rounding per
  operation.
* With ``cfg.adapt`` the evolutions use JADE's adaptation (``oracle.jade``):
  every estimated sample starts a fresh memory (mu_F, mu_CR = F, CR) and an
  empty archive; the draws use the same counter generation codes.
* Semblance calls are counted as the paper counts them (eq.
  ens_semblance): NP_f (1 + NG_f) per estimated sample in stage 0,
  NP_bf (1 + NG_bf) - 1 per estimated sample in a backward or forward stage
  (the own best is not re-evaluated), one per interpolated sample and stage.
"""
from __future__ import annotations

import numpy as np

from . import de as de_mod
from . import jade
from .semblance import semblance_many

f32 = np.float32


def stages(n_cycle: int, n_skip: int):
    """[(kind, direction, init)] for the stage list of Sec. 3.6."""
    out = [("explore", +1, 0)]
    for _ in range(n_cycle):
        out.append(("backward", -1, 0 if n_skip == 0 else 1))
        out.append(("forward", +1, n_skip))
    return out


def estimated(n_t0: int, n_skip: int, init: int):
    return list(range(init, n_t0, n_skip + 1))


def gen_code(stage: int, g: int) -> int:
    return (stage + 1) * 65536 + g


def interpolate(t, est_sorted, theta_of):
    """FP32 linear interpolation in t between the nearest estimated samples."""
    import bisect
    k = bisect.bisect_left(est_sorted, t)
    ta = est_sorted[k - 1] if k > 0 else None
    tb = est_sorted[k] if k < len(est_sorted) else None
    if ta is None:
        return theta_of(tb).copy()
    if tb is None:
        return theta_of(ta).copy()
    w = f32(f32(t - ta) / f32(tb - ta))
    a, b = theta_of(ta), theta_of(tb)
    return (a + f32(w * f32(b - a))).astype(f32)


def ens_search(traces, mid, off, prob, cfg, fitness=None):
    """Run ENS over the m0-major grid of ``prob`` with settings ``cfg``
    (attributes np, ng [= NP_f, NG_f], np_bf, ng_bf, n_skip, n_cycle,
    n_bucket, F, CR, seed, lo, hi). Returns (best_theta, best_S, n_calls).

    ``fitness(theta [n, P, D] float32, domains) -> float32 [n, P]`` gives
    the semblance of each parameter vector at its domain; by default the
    FP64 semblance rounded to FP32. Every decision of the sweep (selection,
    arg-max, keep-if-higher) is taken on these values, so a caller can pass
    another evaluation of the same semblance -- e.g. the FP32 values of an
    implementation under test -- and compare the sweeps step by step on
    identical fitness (FP32 and FP64 semblances round differently and can
    rank two members in opposite orders)."""
    if fitness is None:
        def fitness(theta, domains):
            return semblance_many(traces, mid, off, prob, theta, domains=domains).astype(f32)
    n_m0, n_t0 = prob.n_m0, prob.n_t0
    D = len(cfg.lo)
    lo = np.asarray(cfg.lo, f32)
    hi = np.asarray(cfg.hi, f32)
    n_dom = n_m0 * n_t0
    best_th = np.full((n_dom, D), np.nan, f32)
    best_S = np.full(n_dom, -np.inf, f32)
    n_calls = 0
    nb = cfg.n_bucket
    n_buckets = -(-n_m0 // nb)
    for s, (kind, dirn, init) in enumerate(stages(cfg.n_cycle, cfg.n_skip)):
        NP, NG = (cfg.np, cfg.ng) if kind == "explore" else (cfg.np_bf, cfg.ng_bf)
        est = estimated(n_t0, cfg.n_skip, init)
        est_set = set(est)
        skipped = [t for t in range(n_t0) if t not in est_set]
        for step in range(nb):
            tb = step if dirn > 0 else nb - 1 - step
            snap_th = best_th.copy()
            cmps, prevs = [], []
            for b in range(n_buckets):
                length = min(nb, n_m0 - b * nb)
                if tb >= length:
                    continue
                c = b * nb + tb
                has_prev = 0 <= tb - dirn < length
                cmps.append(c)
                prevs.append(c - dirn if has_prev else -1)
            if not cmps:
                continue
            # estimated samples of every active trace
            doms = [c * n_t0 + t for c in cmps for t in est]
            pop = np.empty((len(doms), NP, D), f32)
            for r, d in enumerate(doms):
                c, t = divmod(d, n_t0)
                cp = prevs[cmps.index(c)]
                seeds = []
                if kind == "explore":
                    if cp >= 0:
                        seeds.append(best_th[cp * n_t0 + t])
                else:
                    if t - 1 >= 0:
                        seeds.append(snap_th[d - 1])
                    if t + 1 < n_t0:
                        seeds.append(snap_th[d + 1])
                    if cp >= 0:
                        seeds.append(best_th[cp * n_t0 + t])
                    seeds.append(snap_th[d])
                seeds = [v for v in seeds if not np.any(np.isnan(v))][:NP]
                for i in range(NP):
                    pop[r, i] = seeds[i] if i < len(seeds) else de_mod.init_individual(
                        cfg.seed, d, i, lo, hi, gen=gen_code(s, 0))
            fit = np.asarray(fitness(pop, doms), f32)
            n_calls += len(doms) * (NP if kind == "explore" else NP - 1)
            adapt = bool(getattr(cfg, "adapt", 0))
            states = [jade.new_state(NP, D, cfg.F, cfg.CR) for _ in doms] if adapt else None
            for g in range(1, NG + 1):
                trial = np.empty_like(pop)
                for r, d in enumerate(doms):
                    if adapt:
                        trial[r], _ = jade.trial_population(states[r], cfg.seed, d, gen_code(s, g),
                                                            pop[r], fit[r], lo, hi)
                    else:
                        trial[r], _ = de_mod.mutate_population(cfg.seed, d, gen_code(s, g),
                                                              pop[r], fit[r], cfg.F, cfg.CR, lo,
                                                              hi)
                tfit = np.asarray(fitness(trial, doms), f32)
                n_calls += len(doms) * NP
                for r, d in enumerate(doms):
                    if adapt:
                        pop[r], fit[r] = jade.select_adapt(states[r], cfg.seed, d, gen_code(s, g),
                                                           pop[r], fit[r], trial[r], tfit[r])
                    else:
                        pop[r], fit[r] = de_mod.select(pop[r], fit[r], trial[r], tfit[r])
            for r, d in enumerate(doms):
                b = de_mod.best_index(fit[r])
                best_th[d], best_S[d] = pop[r, b], fit[r, b]
            # interpolated samples of every active trace
            if skipped:
                idoms = [c * n_t0 + t for c in cmps for t in skipped]
                ith = np.stack([interpolate(d % n_t0, est, lambda tt, c=d // n_t0:
                                            best_th[c * n_t0 + tt]) for d in idoms])
                iS = np.asarray(fitness(ith[:, None, :], idoms), f32)[:, 0]
                n_calls += len(idoms)
                for r, d in enumerate(idoms):
                    if de_mod.rank_key(iS[r]) > de_mod.rank_key(best_S[d]):
                        best_th[d], best_S[d] = ith[r], iS[r]
    return best_th, best_S, n_calls
