"""Checkpoint and resume of a search driven through tt_de_step.

Philox draws are keyed by (seed, domain, generation, individual) and no
generator state exists, so (population, fitness, the trial awaiting
selection and its fitness, the generation number) is the whole state of a
fixed-F/CR search, plus the context's JADE memory and archive for an
adaptive one: saving it to host memory after some generation, creating a
fresh context and continuing from it must give the same bits as an
uninterrupted run.
"""
import numpy as np
import pytest
import torch

import paper_2304_11399_gb300 as tt
from gpu_util import dev, small_line

pytestmark = pytest.mark.gpu


def _generations(ctx, g0, g1, pop, fit, trial, tfit):
    """Generations g0..g1-1 (g0 >= 1); trial/tfit: the pending trial or None."""
    for g in range(g0, g1):
        nxt = torch.empty_like(pop)
        tt.tt_de_step(ctx, g, pop, fit, trial, tfit, nxt)
        trial, tfit = nxt, tt.tt_semblance_eval(ctx, nxt)
    return pop, fit, trial, tfit


def _start(ctx, NP, D):
    pop = torch.empty((ctx.n_dom, NP, D), dtype=torch.float32, device=dev())
    tt.tt_de_step(ctx, 0, pop)
    return pop, tt.tt_semblance_eval(ctx, pop)


@pytest.mark.parametrize("adapt", [0, 1])
def test_resume_is_bit_identical(adapt):
    """adapt = 1 also saves and restores the JADE memory and archive
    (tt_jade_state)."""
    wl = small_line(12, n_cmp=5, ns=120, ap_half=2, np_=24, ng=12, tau_max=0.4)
    wl.de.adapt = adapt
    NP, D = 24, 3
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    pop, fit = _start(ctx, NP, D)
    ref = _generations(ctx, 1, 13, pop, fit, None, None)
    ref = [t.cpu().numpy() for t in ref]
    ctx.close()
    # interrupted after generation 7: state to host, a fresh context, continue
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    pop, fit = _start(ctx, NP, D)
    saved = [t.cpu().numpy().copy() for t in _generations(ctx, 1, 8, pop, fit, None, None)]
    jade = {k: v.cpu() for k, v in tt.tt_jade_state(ctx).items()} if adapt else None
    ctx.close()
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    state = [torch.as_tensor(a, device=dev()) for a in saved]
    if adapt:
        tt.tt_jade_state(ctx, {k: v.to(dev()) for k, v in jade.items()})
    out = [t.cpu().numpy() for t in _generations(ctx, 8, 13, *state)]
    ctx.close()
    for a, b in zip(out, ref):
        np.testing.assert_array_equal(a, b)
