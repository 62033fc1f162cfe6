"""Sharding the search by midpoint slabs, on CPU ranks (gloo).

A line of CMPs is cut into contiguous slabs, one per rank. Each rank holds
only its slab's domains over a copy of the traces its apertures read (the
slab plus a halo of the aperture radius) and runs the oracle's search with
its global domain offset; at every exchange the ranks swap the bests of
their edge rows with the package's halo_exchange (torch.distributed
point-to-point, here over gloo). The slabs together must reproduce the
single-domain oracle search over the whole line bit for bit: parameters,
semblance and call counts, with fixed F, CR and with JADE adaptation, for
two and three ranks (uneven slabs).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _line(adapt):
    from synth import configs
    wl = configs.crs_line(4, n_cmp=7, ns=60, n_events=2, ap_half=2, np_=8, ng=6, exch_every=2,
                          polish_steps=1, tau_max=0.22)
    if adapt:
        wl.de.adapt, wl.de.CR = 1, 0.5
    return wl


def _weights(line):
    """Work per CMP: the trace count of its aperture (clipped at the line ends)."""
    import synth
    return np.diff(synth.line_problem(line, half_window=5, ap_half=2).ap_ptr)


def _worker(rank, world, port, adapt, weighted, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_2304_11399_gb300.slab import halo_exchange
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _line(adapt)
    c0, c1 = synth.slab_bounds(wl.line.n_cmp, world, rank,
                               weights=_weights(wl.line) if weighted else None)
    tr, mid, off, prob, base, has_prev, has_next = synth.slab_problem(
        wl.line, c0, c1, half_window=5, ap_half=2)
    assert (has_prev, has_next) == (rank > 0, rank < world - 1)
    ex = halo_exchange(rank, world)
    n_t0, D = prob.n_t0, 3

    def halo(g, first_row, last_row):
        rows = [torch.from_numpy(np.ascontiguousarray(first_row)),
                torch.from_numpy(np.ascontiguousarray(last_row)),
                torch.zeros((n_t0, D)), torch.zeros((n_t0, D))]
        ex(g, *rows)
        return (rows[2].numpy() if has_prev else None, rows[3].numpy() if has_next else None)

    th, S, n = oracle.search.search(tr, mid, off, prob, wl.de, dom_base=base, halo=halo)
    out[rank] = (th, S, n, c0, c1)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,adapt,weighted", [(2, 0, 0), (3, 0, 0), (2, 1, 0), (3, 0, 1)])
def test_slabs_reproduce_the_whole_line_search(world, adapt, weighted):
    sys.path.insert(0, ROOT)
    import oracle
    wl = _line(adapt)
    th_ref, S_ref, n_ref = oracle.search.search(wl.traces, wl.mid, wl.off, wl.problem, wl.de)
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, adapt, weighted, out), nprocs=world, join=True)
    parts = [out[r] for r in range(world)]
    assert [p[3] for p in parts] == sorted(p[3] for p in parts)
    th = np.concatenate([p[0] for p in parts])
    S = np.concatenate([p[1] for p in parts])
    assert np.array_equal(th, th_ref)
    assert np.array_equal(S, S_ref)
    assert sum(p[2] for p in parts) == n_ref


def test_slab_inputs():
    """Each slab's trace copy holds exactly its apertures' traces (the slab
    plus the aperture halo, clipped at the line ends), in the line's order,
    and its aperture lists name the same traces as the whole-line problem's."""
    sys.path.insert(0, ROOT)
    import synth
    wl = _line(0)
    line = wl.line
    full = synth.line_problem(line, half_window=5, ap_half=2)
    assert synth.slab_bounds(7, 3, 0) == (0, 3) and synth.slab_bounds(7, 3, 2) == (5, 7)
    for world in (1, 2, 3, 7):
        seen = 0
        for r in range(world):
            c0, c1 = synth.slab_bounds(7, world, r)
            tr, mid, off, prob, base, hp, hn = synth.slab_problem(line, c0, c1, half_window=5,
                                                                  ap_half=2)
            assert base == c0 * line.ns and prob.n_m0 == c1 - c0 and (hp, hn) == (c0 > 0, c1 < 7)
            h0 = max(0, c0 - 2) * line.n_off
            assert tr.shape[0] == (min(7, c1 + 2) - max(0, c0 - 2)) * line.n_off
            for k, c in enumerate(range(c0, c1)):
                loc = prob.ap_idx[prob.ap_ptr[k]:prob.ap_ptr[k + 1]]
                glob = full.ap_idx[full.ap_ptr[c]:full.ap_ptr[c + 1]]
                assert np.array_equal(loc + h0, glob)
                assert np.array_equal(tr[loc], line.traces[glob])
            seen += prob.n_dom
        assert seen == line.n_cmp * line.ns


def test_work_weighted_slab_cuts():
    """With per-CMP work weights the slabs are contiguous, non-empty, cover
    the line, and each cut lies where the running work is nearest to its
    share of the total (within half a CMP's weight of it unless a slab would
    be empty); equal weights give the equal-size cut; on the line the edge
    slabs, whose apertures are clipped, take more CMPs than the inner ones
    and the largest slab's work does not exceed that of the equal-size cut."""
    sys.path.insert(0, ROOT)
    import synth
    rng = np.random.default_rng(3)
    for n, world in [(7, 3), (20, 4), (200, 8), (5, 5), (9, 1)]:
        for w in (np.ones(n), rng.uniform(0.5, 2.0, n), np.r_[np.zeros(n - 1), 1.0]):
            cuts = [synth.slab_bounds(n, world, r, weights=w) for r in range(world)]
            assert cuts[0][0] == 0 and cuts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
            assert all(c1 > c0 for c0, c1 in cuts)
            cum = np.concatenate([[0.0], np.cumsum(w)])
            for r in range(1, world):
                k, target = cuts[r][0], r * cum[-1] / world
                clamped = k == cuts[r - 1][0] + 1 or k == n - (world - r)
                assert clamped or abs(cum[k] - target) <= w.max() / 2 + 1e-9
            if np.all(w == 1) and n % world == 0:
                assert cuts == [synth.slab_bounds(n, world, r) for r in range(world)]
    from synth import configs
    big = configs.crs_line(4, n_cmp=200, ns=60, n_events=2, ap_half=10, np_=8, ng=6,
                           exch_every=2, polish_steps=1, tau_max=0.22)
    w = np.diff(big.problem.ap_ptr)
    sizes = [c1 - c0 for c0, c1 in (synth.slab_bounds(200, 8, r, weights=w) for r in range(8))]
    assert sizes[0] > 25 and sizes[-1] > 25 and max(sizes[1:-1]) <= 25
    for world in (4, 8):  # the largest slab's work never grows; at 4 slabs it shrinks
        work = [w[c0:c1].sum() for c0, c1 in (synth.slab_bounds(200, world, r, weights=w)
                                              for r in range(world))]
        eq = [w[c0:c1].sum() for c0, c1 in (synth.slab_bounds(200, world, r)
                                            for r in range(world))]
        assert max(work) < max(eq) if world == 4 else max(work) <= max(eq)
    with pytest.raises(ValueError):
        synth.slab_bounds(3, 4, 0, weights=np.ones(3))


def test_the_halo_rows_matter():
    """Negative control: a slab searched without its neighbours' rows (or
    with the wrong domain offset) does not reproduce its part of the
    whole-line search, so the comparison above checks the exchange."""
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    wl = _line(0)
    th_ref, S_ref, _ = oracle.search.search(wl.traces, wl.mid, wl.off, wl.problem, wl.de)
    c0, c1 = synth.slab_bounds(wl.line.n_cmp, 2, 0)
    tr, mid, off, prob, base, _, _ = synth.slab_problem(wl.line, c0, c1, half_window=5,
                                                        ap_half=2)
    n = prob.n_dom
    th, S, _ = oracle.search.search(tr, mid, off, prob, wl.de, dom_base=base)
    assert not np.array_equal(th, th_ref[:n])
    th2, _, _ = oracle.search.search(tr, mid, off, prob, wl.de, dom_base=base + 1,
                                     halo=lambda g, a, b: (None, np.zeros_like(b)))
    assert not np.array_equal(th2, th_ref[:n])
