"""The search with members evaluated in the order of their window position
(TT_OPT_MEMBER_ORDER = 1; the default orders them when apertures are long)
against the index order: the order only
changes which lane evaluates which member, so best parameters, semblance and
call counts must be identical bit for bit -- on launches that fill the GPU
(the packed kernel) and on small ones (the split kernel), for the CRS, CMP
and FO-CRS operators, BF16-stored traces, JADE adaptation, the moveout form
of long records, and a slab of a sharded line."""
import pytest
import torch

import paper_2304_11399_gb300 as tt
from gpu_util import dev, configs, synth

pytestmark = pytest.mark.gpu


def _search(wl, order, storage="f32", slab=None, **opts):
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, storage=storage,
                           device=dev())
    tt.tt_ctx_set_option(ctx, "member_order", order)
    assert tt.tt_ctx_get_option(ctx, "member_order") == order
    for k, v in opts.items():
        tt.tt_ctx_set_option(ctx, k, v)
    if slab is None:
        th, S, n = tt.tt_search(ctx)
    else:
        th, S, n = tt.tt_search_slab(ctx, *slab)
    out = th.cpu(), S.cpu(), n
    ctx.close()
    return out


def _same(wl, **kw):
    a = _search(wl, True, **kw)
    b = _search(wl, False, **kw)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and a[2] == b[2]
    return a


def _line(seed, n_cmp, **kw):
    kw.setdefault("ns", 200)
    kw.setdefault("n_events", 5)
    kw.setdefault("ap_half", 3)
    kw.setdefault("np_", 64)
    kw.setdefault("ng", 12)
    kw.setdefault("exch_every", 4)
    kw.setdefault("polish_steps", 1)
    kw.setdefault("tau_max", 0.7)
    return configs.crs_line(seed, n_cmp=n_cmp, **kw)


def _launches(wl, order):
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    if order is not None:
        tt.tt_ctx_set_option(ctx, "member_order", order)
    assert tt.tt_ctx_get_option(ctx, "member_order") == ("auto" if order is None else order)
    tt.tt_ctx_set_option(ctx, "search_graph", False)
    tt.tt_ctx_stats(ctx, reset=True)
    tt.tt_search(ctx)
    n = tt.tt_ctx_stats(ctx)["launches"]
    ctx.close()
    return n


def test_automatic_order_follows_the_mean_aperture():
    """The default ("auto") orders the members, one extra launch per
    evaluated population (NG + 1), only when the apertures hold at least 768
    traces on average."""
    for ap_half, n_cmp in ((3, 6), (10, 24)):
        wl = _line(1, n_cmp, ap_half=ap_half, ng=3, exch_every=0, polish_steps=0)
        mean_ap = float((wl.problem.ap_ptr[1:] - wl.problem.ap_ptr[:-1]).mean())
        off, on, auto = (_launches(wl, o) for o in (False, True, None))
        assert on == off + wl.de.ng + 1
        assert auto == (on if mean_ap >= 768 else off)
    assert mean_ap >= 768  # the second line exercises the ordered default
    from paper_2304_11399_gb300 import _lib as L
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    assert ctx.lib.tt_ctx_set_option(ctx.handle, L.TT_OPT_MEMBER_ORDER, 3) == L.TT_ERR_INVALID_ARG
    assert tt.tt_ctx_get_option(ctx, "member_order") == "auto"
    ctx.close()


@pytest.mark.parametrize("kernel", ["packed", "persistent", "scalar"])
def test_crs_line_full_launches(kernel):
    # 30 CMPs x 200 samples x 64 members: 6000 units, above the split threshold
    wl = _line(2, 30)
    th, S, n = _same(wl, kernel=kernel)
    assert n > 0 and bool(torch.isfinite(S).all())


def test_small_launches_split():
    _same(_line(3, 6, np_=24))


def test_odd_population_and_jade():
    wl = _line(4, 8, np_=37)
    wl.de.adapt, wl.de.CR = 1, 0.5
    _same(wl)


def test_bf16_storage_and_cmp_operator():
    _same(_line(5, 10, np_=32), storage="bf16")
    _same(configs.cmp_search(6, ns=300, np_=48, ng=10))


def test_fo_crs():
    _same(configs.fo_panel(7, n_cmp=12, ns=200, n_events=4, np_=40, ng=8, exch_every=4,
                           tau_max=0.7))


def test_moveout_form_and_uneven_apertures():
    # records of up to 3000 samples take the moveout form of the position
    _same(configs.batched(8, n_prob=24, ng=6, domains_per_problem=48))


def test_slab_of_a_sharded_line():
    wl = _line(9, 8, np_=32)
    c0, c1 = synth.slab_bounds(wl.line.n_cmp, 2, 0)
    tr, mid, off, prob, base, hp, hn = synth.slab_problem(wl.line, c0, c1, half_window=5,
                                                          ap_half=3)
    wl.traces, wl.mid, wl.off, wl.problem = tr, mid, off, prob

    def loopback(gen, send_first, send_last, recv_prev, recv_next):
        recv_next.copy_(send_last)

    _same(wl, slab=(base, hp, hn, loopback))
