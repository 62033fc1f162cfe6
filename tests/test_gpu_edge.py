"""Degenerate inputs through the C ABI: a problem with no domains, a context
with no traces (every aperture empty), one-sample records and one-trace
apertures. Nothing may fault; empty work returns empty results, an empty
aperture gives S = 0 and a zero stack, and the ENS sweep without a grid is
rejected with an error."""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_11399_gb300 as tt
from gpu_util import dev, to_dev, synth, configs

pytestmark = pytest.mark.gpu


def _problem(n_dom, ap_ptr, ap_idx, it0, group, n_groups=1, op=1, w=5):
    return synth.Problem(op=op, half_window=w, group_m0=np.zeros(n_groups, np.float32),
                         group_dt=np.full(n_groups, 0.004, np.float32),
                         ap_ptr=np.asarray(ap_ptr, np.int32), ap_idx=np.asarray(ap_idx, np.int32),
                         dom_it0=np.asarray(it0, np.int32), dom_group=np.asarray(group, np.int32))


def _cfg(np_=8, ng=3):
    return configs.DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=1, lo=configs.CRS_LO,
                            hi=configs.CRS_HI, exch_every=0, polish_steps=2, polish_lr=2e-4)


def test_no_domains():
    x = np.random.default_rng(0).standard_normal((4, 50)).astype(np.float32)
    mid, off = np.zeros(4, np.float32), np.arange(4, dtype=np.float32) * 100
    prob = _problem(0, [0, 4], [0, 1, 2, 3], [], [])
    ctx = tt.tt_ctx_create(x, mid, off, prob, _cfg(), device=dev())
    th = torch.empty((0, 3, 3), device=dev())
    assert tt.tt_semblance_eval(ctx, th).shape == (0, 3)
    S, G = tt.tt_semblance_grad(ctx, th)
    assert S.shape == (0, 3) and G.shape == (0, 3, 3)
    assert tt.tt_stack(ctx, torch.empty((0, 3), device=dev())).shape == (0,)
    bt, bs, n = tt.tt_search(ctx)
    assert bt.shape == (0, 3) and bs.shape == (0,) and n == 0
    pop = torch.empty((0, 8, 3), device=dev())
    tt.tt_de_step(ctx, 0, pop)
    with pytest.raises(tt.TTError, match="grid"):
        tt.tt_ens_search(ctx)
    ctx.close()


def test_no_traces_empty_apertures():
    prob = _problem(3, [0, 0], [], [0, 5, 9], [0, 0, 0])
    x = np.zeros((0, 10), np.float32)
    ctx = tt.tt_ctx_create(x, np.zeros(0, np.float32), np.zeros(0, np.float32), prob, _cfg(),
                           device=dev())
    th = to_dev(np.tile(np.array([1e-4, 0.0, 2e-7], np.float32), (3, 2, 1)))
    assert torch.all(tt.tt_semblance_eval(ctx, th) == 0)
    S, G = tt.tt_semblance_grad(ctx, th)
    assert torch.all(S == 0) and torch.all(G == 0)
    assert torch.all(tt.tt_stack(ctx, th[:, 0].contiguous()) == 0)
    bt, bs, n = tt.tt_search(ctx)
    assert torch.all(bs == 0)
    ctx.close()


@pytest.mark.parametrize("w", [0, 3])
def test_one_sample_records_and_one_trace_apertures(w):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 1)).astype(np.float32)
    mid = np.array([0, 12.5, 25], np.float32)
    off = np.array([0, 50, 100], np.float32)
    prob = _problem(4, [0, 1, 3], [1, 0, 2], [0, 0, 0, 0], [0, 1, 1, 0], n_groups=2, w=w)
    theta = np.zeros((4, 3, 3), np.float32)
    theta[:, 1] = [0, 0, 1e-9]
    theta[:, 2] = [1e-3, -1e-7, 0]
    ctx = tt.tt_ctx_create(x, mid, off, prob, None, device=dev())
    S = tt.tt_semblance_eval(ctx, to_dev(theta)).cpu().numpy()
    st = tt.tt_stack(ctx, to_dev(theta[:, 0])).cpu().numpy()
    ctx.close()
    ref = oracle.semblance.semblance_many(x, mid, off, prob, theta)
    assert np.max(np.abs(S - ref)) <= 1e-5
    sref = oracle.stack.stack_many(x, mid, off, prob, theta[:, 0])
    assert np.max(np.abs(st - sref)) <= 1e-6


def test_l1_probe_measures_a_plausible_rate():
    """The L1 probe runs on the context's scratch and reports the bytes it
    loads; its rate is positive and finite, and a fraction of the probe
    (one iteration against many) scales with the bytes."""
    import torch
    import paper_2304_11399_gb300 as tt
    from gpu_util import dev, small_line
    wl = small_line(3, n_cmp=4, ns=80, ap_half=1)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, None, device=dev())
    n_sm = tt.tt_ctx_get_option(ctx, "sm_count")
    assert n_sm == torch.cuda.get_device_properties(dev()).multi_processor_count
    assert tt.tt_ctx_get_option(ctx, "split_max_pairs") == n_sm * 32 * 64
    tt.tt_ctx_probe_l1(ctx, 10)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    n = tt.tt_ctx_probe_l1(ctx, 500)
    b.record()
    torch.cuda.synchronize()
    assert n % (n_sm * 256 * 500 * 32 * 4) == 0 and n <= n_sm * 8 * 256 * 500 * 32 * 4
    rate = n / (a.elapsed_time(b) / 1e3)
    assert np.isfinite(rate) and rate > 0
    assert tt.tt_ctx_probe_l1(ctx, 1) * 500 == n
    with pytest.raises(tt.TTError):
        tt.tt_ctx_probe_l1(ctx, 0)
    ctx.close()
