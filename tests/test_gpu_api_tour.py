"""The public Python API in the order a user calls it, on a small line:
create a context, tune, search, ENS sweep, evaluate a population (plain and
differentiable) and stack along the result. Checks shapes, ranges and the
agreement of the calls with one another (the numerics of each are pinned
against the oracle in the other GPU tests)."""
import numpy as np
import pytest
import torch

import paper_2304_11399_gb300 as tt
from gpu_util import dev, small_line

pytestmark = pytest.mark.gpu


def test_api_tour():
    wl = small_line(2, np_=16, ng=12, exch_every=4, polish_steps=2)
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, wl.de, device=dev())
    n, D = ctx.n_dom, ctx.D
    assert (n, D) == (wl.problem.n_dom, 3)
    th0 = torch.empty((n, wl.de.np, D), device=dev())
    tt.tt_de_step(ctx, 0, th0)
    lo, hi = (torch.tensor(v, device=dev())[:D] for v in (wl.de.lo, wl.de.hi))
    assert bool(((th0 >= lo) & (th0 <= hi)).all())
    times = tt.tt_ctx_autotune(ctx, th0)
    assert len(times) == 6 and all(t > 0 for t in times.values())

    theta, S, n_evals = tt.tt_search(ctx)
    assert theta.shape == (n, D) and S.shape == (n,) and n_evals > 0
    assert bool(((theta >= lo) & (theta <= hi)).all())
    assert bool(((S >= 0) & (S <= 1)).all())
    # the reported S is theta's, within the FP32 bar: the search's launches and this one
    # may take different kernel forms, which sum in different orders
    S_again = tt.tt_semblance_eval(ctx, theta[:, None, :].contiguous())[:, 0]
    assert torch.max(torch.abs(S_again - S)).item() <= 1e-5

    theta_e, S_e, n_e = tt.tt_ens_search(ctx, 5, 1, 5, 1, 2, 1, 4)
    assert theta_e.shape == (n, D) and n_e > 0 and bool(torch.isfinite(S_e).all())
    assert bool(((S_e >= 0) & (S_e <= 1)).all())

    S_pop = tt.tt_semblance_eval(ctx, th0)
    th = th0.clone().requires_grad_()
    S_ad = tt.semblance(ctx, th)
    assert torch.equal(S_ad.detach(), S_pop)
    S_ad.sum().backward()
    assert th.grad.shape == th0.shape and bool(torch.isfinite(th.grad).all())

    stack = tt.tt_stack(ctx, theta)
    assert stack.shape == (n,) and bool(torch.isfinite(stack).all())
    assert np.isfinite(stack.cpu().numpy()).all()
    ctx.close()
