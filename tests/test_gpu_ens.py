"""ENS sweep mode on the GPU (tt_ens_search) against the oracle.

* Call counts equal the oracle's and eq. ens_semblance.
* Without DE generations the sweep is a sequence of Philox draws, seeds,
  arg-maxes and interpolations; the arg-maxes compare semblances that are
  far apart for random parameters, so the GPU and the FP64 oracle must pick
  the same individuals: the bests must agree bit for bit (FP32 seeds, FP32
  interpolation) on nearly every sample.
* The graph-replayed sweep equals the eagerly launched one bit for bit.
* The reported semblance is the oracle's at the reported parameters.
* ENS 5x1 beats JADE 5x1 (tt_search) at about the same number of calls.
* With JADE adaptation inside the sweep the bests still agree with the
  oracle's on nearly every sample.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, synth, configs

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


def _gpu(wl, e, graph=True):
    de = configs.DEConfig(np=max(e.np, e.np_bf), ng=1, F=e.F, CR=e.CR, seed=e.seed, lo=e.lo,
                          hi=e.hi, adapt=e.adapt)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, de, device=dev())
    tt.tt_ctx_set_option(ctx, "search_graph", graph)
    th, S, n = tt.tt_ens_search(ctx, e.np, e.ng, e.np_bf, e.ng_bf, e.n_skip, e.n_cycle,
                                e.n_bucket)
    out = th.cpu().numpy(), S.cpu().numpy(), n
    if graph:  # a second replay of the captured sweep gives the same
        th2, S2, n2 = tt.tt_ens_search(ctx, e.np, e.ng, e.np_bf, e.ng_bf, e.n_skip, e.n_cycle,
                                       e.n_bucket)
        assert np.array_equal(th2.cpu().numpy(), out[0]) and n2 == n
    ctx.close()
    return out


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


@pytest.mark.parametrize("n_skip,nb", [(0, 1), (2, 7)])
def test_no_generation_sweep_matches_oracle_bitwise(n_skip, nb):
    wl = configs.crs_line(2, n_cmp=7, ns=90, n_events=3, ap_half=2, tau_max=0.3)
    e = E(ng=0, ng_bf=0, n_skip=n_skip, n_cycle=1, n_bucket=nb)
    th, S, n = _gpu(wl, e)
    th_o, S_o, n_o = oracle.ens.ens_search(wl.traces, wl.mid, wl.off, wl.problem, e)
    assert n == n_o
    same = np.all(th == th_o, axis=1)
    assert same.mean() >= 0.98, same.mean()
    assert np.max(np.abs(S[same] - S_o[same])) <= 1e-5


def test_adaptive_sweep_matches_oracle():
    """JADE adaptation inside the sweep (5 x 2, 5 x 2): the draws are the
    oracle's bit for bit, so the bests agree wherever the FP32 and FP64
    semblances take the same selection decisions (nearly everywhere)."""
    wl = configs.crs_line(5, n_cmp=6, ns=90, n_events=3, ap_half=2, tau_max=0.3)
    e = E(ng=2, ng_bf=2, n_bucket=3, adapt=1, F=0.5, CR=0.5)
    th, S, n = _gpu(wl, e)
    th_o, S_o, n_o = oracle.ens.ens_search(wl.traces, wl.mid, wl.off, wl.problem, e)
    assert n == n_o
    same = np.all(th == th_o, axis=1)
    assert same.mean() >= 0.9, same.mean()
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, th[:, None, :])
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
