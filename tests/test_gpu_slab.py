"""The search sharded by midpoint slabs (tt_search_slab) on one GPU.

Two or three slabs of a line run as separate contexts, each driven by its
own host thread on its own stream, as one process per GPU would run them;
at every exchange generation the threads swap their edge rows through the
host (the kernels of different slabs never wait on one another; only the
host threads meet). With the small-launch aperture split off -- so that the
semblance of a pair does not depend on the launch size -- the slabs together
give exactly what tt_search gives on the whole line: best parameters,
semblance and call counts, with fixed F, CR and with JADE adaptation.
"""
import threading

import numpy as np
import pytest
import torch

import paper_2304_11399_gb300 as tt
from gpu_util import dev, synth, configs

pytestmark = pytest.mark.gpu


def _line(adapt):
    wl = configs.crs_line(6, n_cmp=9, ns=200, n_events=3, ap_half=3, np_=16, ng=20,
                          exch_every=5, polish_steps=2, tau_max=0.7)
    if adapt:
        wl.de.adapt, wl.de.CR = 1, 0.5
    return wl


def _whole(wl):
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    tt.tt_ctx_set_option(ctx, "split", False)
    th, S, n = tt.tt_search(ctx)
    out = th.cpu().numpy(), S.cpu().numpy(), n
    ctx.close()
    return out


def _slabs(wl, world):
    barrier = threading.Barrier(world, timeout=120)
    rows, results, errors = {}, {}, []

    def run(r):
        try:
            c0, c1 = synth.slab_bounds(wl.line.n_cmp, world, r)
            tr, mid, off, prob, base, hp, hn = synth.slab_problem(wl.line, c0, c1,
                                                                  half_window=5, ap_half=3)
            ctx = tt.tt_ctx_create(tr, mid, off, prob, wl.de, device=dev())
            tt.tt_ctx_set_option(ctx, "split", False)
            s = torch.cuda.Stream(device=dev())

            def exchange(gen, send_first, send_last, recv_prev, recv_next):
                s.synchronize()
                rows[(r, gen)] = (send_first.cpu(), send_last.cpu())
                barrier.wait()
                if hp:
                    recv_prev.copy_(rows[(r - 1, gen)][1])
                if hn:
                    recv_next.copy_(rows[(r + 1, gen)][0])
                s.synchronize()
                barrier.wait()

            with torch.cuda.stream(s):
                th, S, n = tt.tt_search_slab(ctx, base, hp, hn, exchange, stream=s)
            s.synchronize()
            results[r] = (th.cpu().numpy(), S.cpu().numpy(), n)
            ctx.close()
        except BaseException as e:  # reported by the main thread
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return [results[r] for r in range(world)]


@pytest.mark.parametrize("world,adapt", [(2, 0), (3, 0), (2, 1)])
def test_slabs_equal_the_whole_line_search(world, adapt):
    wl = _line(adapt)
    th_ref, S_ref, n_ref = _whole(wl)
    parts = _slabs(wl, world)
    assert np.array_equal(np.concatenate([p[0] for p in parts]), th_ref)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), S_ref)
    assert sum(p[2] for p in parts) == n_ref


def test_slab_without_neighbours_is_the_plain_search():
    """One slab covering the whole line (no neighbours, dom_base 0) is
    tt_search itself, split on or off."""
    wl = _line(0)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    th, S, n = tt.tt_search(ctx)
    th2, S2, n2 = tt.tt_search_slab(ctx, 0, False, False)
    assert torch.equal(th, th2) and torch.equal(S, S2) and n == n2
    ctx.close()


def test_slab_argument_checks():
    wl = _line(0)
    c0, c1 = synth.slab_bounds(wl.line.n_cmp, 2, 0)
    tr, mid, off, prob, base, hp, hn = synth.slab_problem(wl.line, c0, c1, half_window=5,
                                                          ap_half=3)
    ctx = tt.tt_ctx_create(tr, mid, off, prob, wl.de, device=dev())
    with pytest.raises(tt.TTError, match="needs exchange"):
        tt.tt_search_slab(ctx, base, hp, hn, None)
    with pytest.raises(tt.TTError, match="dom_base"):
        tt.tt_search_slab(ctx, -1, False, False)

    def failing(gen, *rows):
        raise RuntimeError("transport down")

    with pytest.raises(RuntimeError, match="transport down"):
        tt.tt_search_slab(ctx, base, hp, hn, failing)
    ctx.close()
