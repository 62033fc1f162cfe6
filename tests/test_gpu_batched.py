"""Batched uneven problems, kernel variants, autotuner and the CUDA-graph
search.

Packed problems: many independent CRS problems with 16-240 traces and
750-3000 samples at 2 or 4 ms each, in one context and one launch per
generation. Every semblance kernel variant (packed grid, persistent queue,
scalar; 128 or 256 threads) performs the same operations in the same order,
so they must agree bit for bit; small launches run the aperture-split kernel
under every variant (bit for bit the same again, within 1e-5 of the oracle);
the graph-replayed search must equal the eagerly launched one bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from paper_2304_11399_gb300 import _lib
from gpu_util import dev, random_theta, to_dev, small_line, synth, configs

pytestmark = pytest.mark.gpu
VARIANTS = _lib.TUNE_CANDIDATES


def _all_variants(ctx, theta):
    """S from the six one-warp-per-unit variants (split off) and, under key
    "split", from the aperture-split small-launch kernel of every variant."""
    out, split = {}, []
    for kern, block in VARIANTS:
        tt.tt_ctx_set_option(ctx, "kernel", kern)
        tt.tt_ctx_set_option(ctx, "block", block)
        tt.tt_ctx_set_option(ctx, "split", False)
        out[(kern, block)] = tt.tt_semblance_eval(ctx, theta).cpu().numpy()
        tt.tt_ctx_set_option(ctx, "split", True)
        split.append(tt.tt_semblance_eval(ctx, theta).cpu().numpy())
    tt.tt_ctx_set_option(ctx, "kernel", "packed")
    tt.tt_ctx_set_option(ctx, "block", 256)
    n_pairs = split[0].size
    if n_pairs < tt.tt_ctx_get_option(ctx, "split_max_pairs"):
        for v in split[1:]:
            assert np.array_equal(v, split[0])
    else:  # too many pairs to split: the option changes nothing
        for k, v in zip(VARIANTS, split):
            assert np.array_equal(v, out[k])
    out["split"] = split[0]
    return out


@pytest.fixture(scope="module")
def batch():
    return configs.batched(3, n_prob=40, ng=80, domains_per_problem=48)


@pytest.mark.parametrize("P", [1, 4, 20, 64, 130])
def test_variants_bit_identical_on_a_line(P):
    """2400 domains: P = 1 (38 units) splits the aperture over 9 blocks of 8
    warps per unit, P = 4 (150 units) over 7 blocks of 8 warps, P = 20 (750
    units) over 2 blocks of 8 warps, P = 64 (2400 units) over one block of 8
    warps,
    P = 130 (4875 units) is too large to split; the oracle checks a sample
    of domains for the two largest P."""
    wl = small_line(31)
    theta = random_theta(wl.problem.n_dom, P, wl.de.lo, wl.de.hi, P)
    doms = np.arange(wl.problem.n_dom)
    if P >= 64:
        doms = np.sort(np.random.default_rng(P).choice(doms, 300, replace=False))
    ora = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, theta[doms],
                                          domains=doms)
    for storage, tol in (("f32", 1e-5), ("bf16", 2e-3)):
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, storage=storage,
                               device=dev())
        res = _all_variants(ctx, to_dev(theta))
        ctx.close()
        ref = res[("packed", 256)]
        for k in VARIANTS:
            assert np.array_equal(res[k], ref), (storage, k)
        assert np.max(np.abs(ref[doms] - ora)) <= tol
        assert np.max(np.abs(res["split"][doms] - ora)) <= tol


def test_batched_uneven_parity_all_variants(batch):
    wl = batch
    prob = wl.problem
    theta = random_theta(prob.n_dom, 16, wl.de.lo, wl.de.hi, 7)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    res = _all_variants(ctx, to_dev(theta))
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta)
    for k in VARIANTS:
        assert np.array_equal(res[k], res[("packed", 256)]), k
    assert np.max(np.abs(res[("packed", 256)] - ref)) <= 1e-5
    assert np.max(np.abs(res["split"] - ref)) <= 1e-5
    times = tt.tt_ctx_autotune(ctx, to_dev(theta))
    assert set(times) == set(VARIANTS) and all(t > 0 for t in times.values())
    best = min(times, key=times.get)
    if best[0] == "persistent":  # kept only when more than 3% ahead of the rest
        alt = min((k for k in times if k[0] != "persistent"), key=times.get)
        if times[alt] <= times[best] * (1 + np.float32(0.03)):
            best = alt
    assert (tt.tt_ctx_get_option(ctx, "kernel"), tt.tt_ctx_get_option(ctx, "block")) == best
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    assert np.array_equal(S, res["split"])  # a small launch: split by default
    ctx.close()


def test_graph_search_equals_eager_search():
    wl = configs.crs_line(4, n_cmp=8, ns=240, n_events=3, ap_half=3, np_=24, ng=25,
                          exch_every=5, polish_steps=3, tau_max=0.8)
    out = {}
    for graph in (False, True):
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
        tt.tt_ctx_set_option(ctx, "search_graph", graph)
        runs = []
        for _ in range(2):  # graph: capture + replay, then a second replay
            tt.tt_ctx_stats(ctx, reset=True)
            bt, bs, n = tt.tt_search(ctx)
            st = tt.tt_ctx_stats(ctx)
            runs.append((bt.cpu().numpy(), bs.cpu().numpy(), n, st["launches"]))
        ctx.close()
        out[graph] = runs
    for graph in (False, True):
        for r in out[graph]:
            np.testing.assert_array_equal(r[0], out[False][0][0])
            np.testing.assert_array_equal(r[1], out[False][0][1])
            assert r[2] == out[False][0][2] and r[3] == out[False][0][3]


def test_persistent_graph_search_on_batched_problems():
    """24 problems, every sample a domain, DE 64 x 80, persistent kernel in
    a graph: recovery of isolated strong events' recentred parameters (the
    problems' reference midpoint is 0) and oracle re-evaluation."""
    wl = configs.batched(5, n_prob=24, ng=80)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    tt.tt_ctx_set_option(ctx, "kernel", "persistent")
    bt, bs, n = tt.tt_search(ctx)
    bt, bs = bt.cpu().numpy(), bs.cpu().numpy()
    ctx.close()
    assert n == oracle.counts.search_calls(prob.n_dom, 64, 80, 0, 0)
    rng = np.random.default_rng(0)
    doms = rng.choice(prob.n_dom, 300, replace=False)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, bt[doms][:, None, :],
                                          domains=doms)[:, 0]
    assert np.max(np.abs(ref - bs[doms])) <= 1e-5
    first = np.searchsorted(prob.dom_group, np.arange(prob.n_groups))
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    tried = hits = 0
    for p in range(prob.n_groups):
        ev = wl.info["events"][p]
        dt = float(prob.group_dt[p])
        for e in range(len(ev)):
            others = np.delete(ev[:, 1], e)
            if abs(ev[e, 5]) < 0.7 or np.any(np.abs(others - ev[e, 1]) < 0.1):
                continue
            truth = synth.crs_recentre(ev[e], 0.0)
            it = int(round(truth[0] / dt))
            if wl.info["ntr"][p] < 48 or not (lo[2] < truth[3] < hi[2]):
                continue
            d = first[p] + it
            tried += 1
            hits += int(bt[d, 2] == pytest.approx(truth[3], rel=0.01))
    assert tried >= 10 and hits >= 0.8 * tried, (hits, tried)


@pytest.mark.slow
def test_full_batched_workload():
    """4096 problems (every sample a domain, ~7.7M domains), DE 64 x 80,
    autotuned kernel, graph-replayed search; oracle re-evaluation of 1000
    sampled domains."""
    import time
    wl = configs.batched(0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    theta = torch.empty((prob.n_dom, 64, 3), device=dev())
    tt.tt_de_step(ctx, 0, theta)
    times = tt.tt_ctx_autotune(ctx, theta)
    del theta
    bt, bs, n = tt.tt_search(ctx)  # capture + first replay
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt, bs, n = tt.tt_search(ctx)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ctx.close()
    print(f"batched 4096: {prob.n_dom} domains, {secs:.2f} s per search, "
          f"{prob.n_dom / secs:.0f} ZO samples/s, tune {times}")
    assert n == oracle.counts.search_calls(prob.n_dom, 64, 80, 0, 0)
    bt, bs = bt.cpu().numpy(), bs.cpu().numpy()
    doms = np.random.default_rng(1).choice(prob.n_dom, 1000, replace=False)
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, bt[doms][:, None, :],
                                          domains=doms)[:, 0]
    assert np.max(np.abs(ref - bs[doms])) <= 1e-5


@pytest.mark.slow
def test_full_batched_workload_sampled_outputs():
    """The 4096-problem batched workload at full size (7.6M domains), NP = 64
    random vectors at every domain in the launch configuration the bench
    times (autotuned variant): 300 sampled domains recomputed by the oracle."""
    wl = configs.batched(0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev())
    th = torch.empty((prob.n_dom, 64, 3), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, th)
    tt.tt_ctx_autotune(ctx, th)
    S = tt.tt_semblance_eval(ctx, th).cpu().numpy()
    ctx.close()
    doms = np.sort(np.random.default_rng(5).choice(prob.n_dom, 300, replace=False))
    theta = th[torch.as_tensor(doms, device=dev())].cpu().numpy()
    ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob, theta, domains=doms)
    assert np.max(np.abs(S[doms] - ref)) <= 1e-5
    assert np.all((S >= 0) & (S <= 1 + 1e-6))
