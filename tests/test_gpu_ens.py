"""ENS sweep mode on the GPU (tt_ens_search) against the oracle.

* Call counts equal the oracle's and eq. ens_semblance.
* Step-local parity: the oracle's sweep, fed the GPU's own FP32 semblance
  values as its fitness, takes every decision the GPU takes -- seeds,
  random members, DE selections, arg-maxes, interpolations and the
  keep-if-higher rule -- so the bests and their semblances agree bit for
  bit on every sample, with fixed F and CR and with JADE adaptation. (FP32
  and FP64 semblances round differently and may rank two members in
  opposite orders, which is why the FP64 oracle's own fitness is not used
  for this comparison; the reported semblance is checked against the FP64
  oracle separately, within 1e-5.)
* The graph-replayed sweep equals the eagerly launched one bit for bit.
* ENS 5x1 beats JADE 5x1 (tt_search) at about the same number of calls.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, to_dev, synth, configs

pytestmark = pytest.mark.gpu


@dataclasses.dataclass
class E:
    np: int = 5
    ng: int = 1
    np_bf: int = 5
    ng_bf: int = 1
    n_skip: int = 2
    n_cycle: int = 1
    n_bucket: int = 8
    F: float = 0.5
    CR: float = 0.9
    seed: int = 11
    lo: tuple = configs.CRS_LO
    hi: tuple = configs.CRS_HI
    adapt: int = 0


def _gpu(wl, e, graph=True, split=True):
    de = configs.DEConfig(np=max(e.np, e.np_bf), ng=1, F=e.F, CR=e.CR, seed=e.seed, lo=e.lo,
                          hi=e.hi, adapt=e.adapt)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, de, device=dev())
    tt.tt_ctx_set_option(ctx, "search_graph", graph)
    tt.tt_ctx_set_option(ctx, "split", split)
    th, S, n = tt.tt_ens_search(ctx, e.np, e.ng, e.np_bf, e.ng_bf, e.n_skip, e.n_cycle,
                                e.n_bucket)
    out = th.cpu().numpy(), S.cpu().numpy(), n
    if graph:  # a second replay of the captured sweep gives the same
        th2, S2, n2 = tt.tt_ens_search(ctx, e.np, e.ng, e.np_bf, e.ng_bf, e.n_skip, e.n_cycle,
                                       e.n_bucket)
        assert np.array_equal(th2.cpu().numpy(), out[0]) and n2 == n
    ctx.close()
    return out


def _gpu_fitness(wl):
    """The GPU's FP32 semblance of each parameter vector at its domain, from
    tt_semblance_eval with the aperture split off. Without the split, the
    semblance of a (vector, domain) pair is one thread's sum over the
    aperture in entry order, the same bits in every launch of every kernel
    variant, so these are exactly the values a sweep run with the split off
    takes its decisions on."""
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, None, device=dev())
    tt.tt_ctx_set_option(ctx, "split", False)
    n_dom = wl.problem.n_dom

    def fitness(theta, domains):
        d = np.asarray(domains)
        full = np.zeros((n_dom,) + theta.shape[1:], np.float32)
        full[d] = theta
        return tt.tt_semblance_eval(ctx, to_dev(full)).cpu().numpy()[d]

    return ctx, fitness


@pytest.mark.parametrize("n_skip,n_cycle,nb,n_m0", [(2, 1, 4, 6), (1, 2, 3, 5), (0, 1, 6, 6)])
def test_counts_match_oracle_and_paper(n_skip, n_cycle, nb, n_m0):
    wl = configs.crs_line(1, n_cmp=n_m0, ns=60, n_events=2, ap_half=2, tau_max=0.2)
    e = E(n_skip=n_skip, n_cycle=n_cycle, n_bucket=nb)
    th, S, n = _gpu(wl, e)
    _, _, n_ref = oracle.ens.ens_search(wl.traces, wl.mid, wl.off, wl.problem, e)
    assert n == n_ref == oracle.counts.ens_calls(wl.problem.n_dom, 5, 1, 5, 1, n_skip, n_cycle)
    assert not np.any(np.isnan(th))
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, th[:, None, :])
    assert np.max(np.abs(ref[:, 0] - S)) <= 1e-5


@pytest.mark.parametrize("ng,n_skip,n_cycle,nb,adapt", [
    (0, 0, 1, 1, 0), (0, 2, 1, 7, 0), (2, 2, 1, 3, 0), (1, 1, 2, 4, 0), (3, 0, 1, 7, 0),
    (2, 2, 1, 3, 1), (1, 1, 2, 7, 1)])
def test_sweep_matches_oracle_step_local(ng, n_skip, n_cycle, nb, adapt):
    """Every best, and the semblance reported with it, equals the oracle's
    sweep bit for bit when both decide on the GPU's FP32 fitness: no
    generations (seeds, random members, arg-maxes and interpolations only),
    DE generations with fixed F and CR, and JADE adaptation; several N_skip,
    N_cycle and bucket sizes (ragged last bucket included)."""
    wl = configs.crs_line(2, n_cmp=7, ns=90, n_events=3, ap_half=2, tau_max=0.3)
    e = E(ng=ng, ng_bf=ng, n_skip=n_skip, n_cycle=n_cycle, n_bucket=nb, adapt=adapt,
          CR=0.5 if adapt else 0.9)
    th, S, n = _gpu(wl, e, split=False)
    ctx, fitness = _gpu_fitness(wl)
    th_o, S_o, n_o = oracle.ens.ens_search(wl.traces, wl.mid, wl.off, wl.problem, e,
                                           fitness=fitness)
    ctx.close()
    assert n == n_o
    assert not np.any(np.isnan(th)) and not np.any(np.isnan(th_o))
    assert np.array_equal(th, th_o), int(np.sum(np.any(th != th_o, axis=1)))
    assert np.array_equal(S, S_o)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, th[:, None, :])
    assert np.max(np.abs(ref[:, 0] - S)) <= 1e-5


def test_split_sweep_reports_exact_semblance():
    """With the aperture split on (the default; its rounding differs from
    the one-thread sum), the reported semblance is still the FP64 oracle's
    at the reported parameters within 1e-5, with and without adaptation."""
    wl = configs.crs_line(5, n_cmp=6, ns=90, n_events=3, ap_half=2, tau_max=0.3)
    for adapt in (0, 1):
        e = E(ng=2, ng_bf=2, n_bucket=3, adapt=adapt, F=0.5, CR=0.5 if adapt else 0.9)
        th, S, n = _gpu(wl, e)
        assert n == oracle.counts.ens_calls(wl.problem.n_dom, 5, 2, 5, 2, 2, 1)
        ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem,
                                              th[:, None, :])
        assert np.max(np.abs(ref[:, 0] - S)) <= 1e-5


def test_graph_equals_eager():
    wl = configs.crs_line(3, n_cmp=9, ns=120, n_events=3, ap_half=2, tau_max=0.4)
    e = E(n_bucket=5)
    a = _gpu(wl, e, graph=False)
    b = _gpu(wl, e, graph=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_ens_beats_jade_at_equal_cost():
    wl = configs.crs_line(7, n_cmp=32, ns=300, n_events=4, ap_half=3, snr=8.0, tau_max=1.0)
    prob = synth.line_problem(wl.line, half_window=5, ap_half=3)
    wl.problem = prob
    th_e, S_e, n_e = _gpu(wl, E(n_bucket=32))
    jade = configs.DEConfig(np=5, ng=1, F=0.5, CR=0.9, seed=11, lo=configs.CRS_LO,
                            hi=configs.CRS_HI)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, jade, device=dev())
    th_j, S_j, n_j = tt.tt_search(ctx)
    S_j = S_j.cpu().numpy()
    ctx.close()
    assert abs(n_e - n_j) / n_j < 0.15
    assert float(np.sqrt(np.mean(S_e ** 2))) > 1.5 * float(np.sqrt(np.mean(S_j ** 2)))


@pytest.mark.slow
def test_full_line_sweep_in_the_bench_configuration():
    """The sweep the bench times on the full CRS line (300,000 domains,
    NP 5 x NG 1 both ways, N_skip 2, N_cycle 1, buckets of 64 traces):
    call count, every sample reached, and the reported S equal to the
    oracle's at the reported parameters on 300 sampled domains."""
    wl = configs.crs_line(0)
    prob = wl.problem
    th, S, n = _gpu(wl, E(n_bucket=64))
    assert n == oracle.counts.ens_calls(prob.n_dom, 5, 1, 5, 1, 2, 1)
    assert not np.any(np.isnan(th)) and np.all((S >= 0) & (S <= 1 + 1e-6))
    doms = np.sort(np.random.default_rng(8).choice(prob.n_dom, 300, replace=False))
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, th[doms][:, None, :],
                                          domains=doms)[:, 0]
    assert np.max(np.abs(ref - S[doms])) <= 1e-5
