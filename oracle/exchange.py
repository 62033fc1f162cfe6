"""Neighbour exchange of best individuals (TEST INFRASTRUCTURE).

Evolution by neighborhood similarity (Sec. 3.2 "Similarities between
neighboring domains", Sec. 3.3 "Information propagation", Sec. 3.6): the
best individual of a domain is introduced into the populations of the
neighbouring zero-offset samples, i.e. the time samples above and below on
the same trace and the same time sample on the adjacent traces (the four
seeds of the backward step, Sec. 3.3), where it replaces a member.

Readings taken here (the paper gives the sweep, not a synchronous rule):
* Domains form an (m0, t0) grid laid out m0-major, d = im0 * n_t0 + it0.
* The neighbours of (im0, it0), in this order, are (im0, it0-1),
  (im0, it0+1), (im0-1, it0), (im0+1, it0); those off the grid are absent.
* Every domain reads a snapshot of all bests taken before the exchange, so
  the result does not depend on the order domains are processed in.
* The q-th present neighbour's best replaces the q-th worst member, ranked
  by (semblance ascending, index ascending) over the members other than
  the domain's own best (argmax, lowest index on ties), so the domain's own
  best is kept as the fourth seed of Sec. 3.3. Its semblance is then
  evaluated at the receiving domain.
"""
from __future__ import annotations

import numpy as np

from .de import best_index, rank_key


def neighbours(d: int, n_m0: int, n_t0: int, has_prev: bool = False, has_next: bool = False):
    """Present neighbours of domain d in the fixed order (t-1, t+1, m-1, m+1).

    When the grid is one slab of a longer line, the m0 rows just before and
    after it belong to the neighbouring slabs: with has_prev (has_next) the
    neighbour (m-1) of the first row ((m+1) of the last row) is present and
    returned as ("prev", it) (("next", it)), its best coming from that slab."""
    im, it = divmod(d, n_t0)
    out = []
    if it > 0:
        out.append(d - 1)
    if it < n_t0 - 1:
        out.append(d + 1)
    if im > 0:
        out.append(d - n_t0)
    elif has_prev:
        out.append(("prev", it))
    if im < n_m0 - 1:
        out.append(d + n_t0)
    elif has_next:
        out.append(("next", it))
    return out


def worst_slots(fit, exclude: int, n: int):
    """The n worst members by (fitness ascending, index ascending), skipping
    ``exclude``."""
    order = sorted((i for i in range(len(fit)) if i != exclude),
                   key=lambda i: (rank_key(fit[i]), i))
    return order[:n]


def exchange_plan(n_m0, n_t0, pop, fit, best_theta, halo_prev=None, halo_next=None):
    """imports [n_dom, 4, D] (zeros where absent) and slots [n_dom, 4] (-1
    absent). halo_prev / halo_next [n_t0, D], if given, are the snapshot
    bests of the m0 rows just before / after the grid (neighbouring slabs)."""
    n_dom, NP, D = pop.shape
    imports = np.zeros((n_dom, 4, D), np.float32)
    slots = np.full((n_dom, 4), -1, np.int32)
    for d in range(n_dom):
        nb = neighbours(d, n_m0, n_t0, halo_prev is not None, halo_next is not None)
        ws = worst_slots(fit[d], best_index(fit[d]), len(nb))
        for q, (e, s) in enumerate(zip(nb, ws)):
            if isinstance(e, tuple):
                imports[d, q] = (halo_prev if e[0] == "prev" else halo_next)[e[1]]
            else:
                imports[d, q] = best_theta[e]
            slots[d, q] = s
    return imports, slots


def apply_exchange(pop, fit, imports, slots, import_fit):
    """Write the imports and their semblance into their slots."""
    pop, fit = pop.copy(), fit.copy()
    for d in range(pop.shape[0]):
        for q in range(4):
            s = slots[d, q]
            if s >= 0:
                pop[d, s] = imports[d, q]
                fit[d, s] = import_fit[d, q]
    return pop, fit


def best_snapshot(pop, fit):
    """best_theta[d] = pop[d, argmax fit[d]]."""
    return np.stack([pop[d, best_index(fit[d])] for d in range(pop.shape[0])])
