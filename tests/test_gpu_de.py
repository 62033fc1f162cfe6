"""GPU DE step, best snapshot and neighbour exchange against the oracle.

Random draws, mutation indices, crossover masks, selections and argmaxes are
integer decisions and must match bit for bit; the trial vectors are FP32
with one rounding per operation on both sides, so they match bit for bit
too. The oracle is fed the same fitness arrays as the kernel.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, random_theta, to_dev, small_line, configs

pytestmark = pytest.mark.gpu
f32 = np.float32


def _ctx(n_dom_grid=(3, 7), NP=16, op=1, seed=123, F=0.5, CR=0.9):
    wl = small_line(0, n_cmp=n_dom_grid[0], ns=n_dom_grid[1] + 20, ap_half=1, np_=NP,
                    t0_range=(10, 10 + n_dom_grid[1]))
    wl.de.seed, wl.de.F, wl.de.CR = seed, F, CR
    if op == 0:
        wl.problem.op = 0
        wl.de.lo, wl.de.hi = (configs.C_BOUNDS_CMP[0],), (configs.C_BOUNDS_CMP[1],)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    return ctx, wl


def _fit(rng, shape, ties=True, nans=True):
    f = rng.uniform(0, 1, shape).astype(f32)
    if ties:
        f[..., 3] = f[..., 1]
        f[0, :] = 0.25
    if nans:
        f[1, 2] = np.nan
        f[2, :] = np.nan
    return f


@pytest.mark.parametrize("op,NP,seed", [(1, 16, 1), (1, 37, 2), (0, 33, 3), (1, 64, 2 ** 40 + 7),
                                        (1, 1024, 5)])
def test_init_and_step_bit_exact(op, NP, seed):
    ctx, wl = _ctx(NP=NP, op=op, seed=seed)
    D = ctx.D
    n = ctx.n_dom
    lo, hi = np.array(wl.de.lo, f32), np.array(wl.de.hi, f32)
    pop = torch.empty((n, NP, D), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, pop)
    ref0 = oracle.de.de_step(0, np.zeros((n, NP, D), f32), None, None, None, seed, wl.de.F,
                             wl.de.CR, lo, hi)[0]
    np.testing.assert_array_equal(pop.cpu().numpy(), ref0)
    rng = np.random.default_rng(seed % 1000)
    fit = _fit(rng, (n, NP))
    trial = random_theta(n, NP, lo, hi, 77)
    tfit = _fit(rng, (n, NP), ties=False)
    tfit[:, 1] = fit[:, 1]                       # equal fitness: the child wins
    for g in (1, 2, 57):
        p_t, f_t = to_dev(ref0), to_dev(fit)
        nxt = torch.empty_like(p_t)
        best = torch.empty((n,), dtype=torch.int32, device=dev())
        tt.tt_de_step(ctx, g, p_t, f_t, to_dev(trial), to_dev(tfit), nxt, best)
        rp, rf, rn, rb = oracle.de.de_step(g, ref0, fit, trial, tfit, seed, wl.de.F, wl.de.CR,
                                           lo, hi)
        np.testing.assert_array_equal(p_t.cpu().numpy(), rp)
        np.testing.assert_array_equal(f_t.cpu().numpy(), rf)
        np.testing.assert_array_equal(best.cpu().numpy(), rb)
        np.testing.assert_array_equal(nxt.cpu().numpy(), rn)
    ctx.close()


def test_select_only_and_mutate_only_modes():
    ctx, wl = _ctx(NP=20, seed=9)
    n, NP, D = ctx.n_dom, 20, 3
    lo, hi = np.array(wl.de.lo, f32), np.array(wl.de.hi, f32)
    rng = np.random.default_rng(1)
    pop = random_theta(n, NP, lo, hi, 1)
    fit = _fit(rng, (n, NP))
    trial = random_theta(n, NP, lo, hi, 2)
    tfit = _fit(rng, (n, NP), ties=False, nans=False)
    p_t, f_t = to_dev(pop), to_dev(fit)
    best = torch.empty((n,), dtype=torch.int32, device=dev())
    tt.tt_de_step(ctx, 4, p_t, f_t, to_dev(trial), to_dev(tfit), None, best)
    rp, rf, _, rb = oracle.de.de_step(4, pop, fit, trial, tfit, 9, 0.5, 0.9, lo, hi, mutate=False)
    np.testing.assert_array_equal(p_t.cpu().numpy(), rp)
    np.testing.assert_array_equal(best.cpu().numpy(), rb)
    nxt = torch.empty_like(p_t)
    tt.tt_de_step(ctx, 5, p_t, f_t, None, None, nxt)
    _, _, rn, _ = oracle.de.de_step(5, rp, rf, None, None, 9, 0.5, 0.9, lo, hi)
    np.testing.assert_array_equal(nxt.cpu().numpy(), rn)
    ctx.close()


@pytest.mark.parametrize("F,CR", [(0.0, 0.0), (1.0, 1.0), (0.5, 0.3), (2.0, 0.9)])
def test_control_parameter_extremes(F, CR):
    ctx, wl = _ctx(NP=12, seed=17, F=F, CR=CR)
    n, NP, D = ctx.n_dom, 12, 3
    lo, hi = np.array(wl.de.lo, f32), np.array(wl.de.hi, f32)
    pop = random_theta(n, NP, lo, hi, 3)
    fit = np.random.default_rng(3).uniform(0, 1, (n, NP)).astype(f32)
    nxt = torch.empty((n, NP, D), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 3, to_dev(pop), to_dev(fit), None, None, nxt)
    _, _, rn, _ = oracle.de.de_step(3, pop, fit, None, None, 17, F, CR, lo, hi)
    np.testing.assert_array_equal(nxt.cpu().numpy(), rn)
    assert np.all(rn >= lo) and np.all(rn <= hi)
    ctx.close()


def test_best_snapshot():
    ctx, wl = _ctx(NP=40)
    n = ctx.n_dom
    rng = np.random.default_rng(4)
    pop = random_theta(n, 40, wl.de.lo, wl.de.hi, 4)
    fit = _fit(rng, (n, 40))
    bt, bs = tt.tt_best_snapshot(ctx, to_dev(pop), to_dev(fit))
    snap = oracle.exchange.best_snapshot(pop, fit)
    np.testing.assert_array_equal(bt.cpu().numpy(), snap)
    b = [oracle.de.best_index(fit[d]) for d in range(n)]
    np.testing.assert_array_equal(bs.cpu().numpy(), fit[np.arange(n), b])
    ctx.close()


@pytest.mark.parametrize("grid,NP", [((3, 7), 16), ((1, 9), 5), ((4, 1), 8), ((2, 5), 100)])
def test_neighbor_exchange(grid, NP):
    ctx, wl = _ctx(n_dom_grid=grid, NP=NP)
    n, D = ctx.n_dom, 3
    rng = np.random.default_rng(5)
    pop = random_theta(n, NP, wl.de.lo, wl.de.hi, 5)
    fit = _fit(rng, (n, NP), nans=n > 2)
    snap = oracle.exchange.best_snapshot(pop, fit)
    p_t, f_t = to_dev(pop), to_dev(fit)
    imports, slots = tt.tt_neighbor_exchange(ctx, grid[0], grid[1], to_dev(snap), p_t, f_t)
    torch.cuda.synchronize()
    ri, rs = oracle.exchange.exchange_plan(grid[0], grid[1], pop, fit, snap)
    np.testing.assert_array_equal(slots.cpu().numpy(), rs)
    np.testing.assert_array_equal(imports.cpu().numpy(), ri)
    ifit = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, wl.problem, ri)
    rp, rf = oracle.exchange.apply_exchange(pop, fit, ri, rs, ifit.astype(f32))
    np.testing.assert_array_equal(p_t.cpu().numpy(), rp)
    got = f_t.cpu().numpy()
    moved = np.zeros_like(got, bool)
    for d in range(n):
        for q in range(4):
            if rs[d, q] >= 0:
                moved[d, rs[d, q]] = True
    np.testing.assert_array_equal(got[~moved], rf[~moved])
    assert np.max(np.abs(got[moved] - rf[moved])) <= 1e-5
    ctx.close()


def test_exchange_rejects_wrong_grid():
    ctx, wl = _ctx()
    z = torch.zeros((ctx.n_dom, 16, 3), device=dev())
    with pytest.raises(tt.TTError, match="n_m0"):
        tt.tt_neighbor_exchange(ctx, 2, 2, torch.zeros((ctx.n_dom, 3), device=dev()), z,
                                torch.zeros((ctx.n_dom, 16), device=dev()))
    ctx.close()
