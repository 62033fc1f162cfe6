"""Stacked zero-offset output along an operator (TEST INFRASTRUCTURE).

Sec. 1: a traveltime operator rebuilds the zero-offset sample from the
amplitudes of the traces it crosses, which is what enhances the signal-to-
noise ratio; Sec. 5.1 shows the resulting stacking panels. The paper prints
no stacking formula. The reading adopted here is the plain stack of the
operator's amplitudes:

    stack(m0, t0; theta) = (1/N) sum_i a_i0,

where a_i0 is the amplitude of aperture trace i at the operator's traveltime
t_i, read by the same linear interpolation as the centre sample (k = 0) of
the semblance window (``oracle.semblance``): a trace with T < 0 adds zero and
still counts in N, and an empty aperture stacks to 0. FP64 throughout.
"""
from __future__ import annotations

import numpy as np

from .semblance import traveltime_sq, window_amplitudes, domain_data


def stack(x, dt, dm, h, t0, op, theta) -> float:
    """Mean centre amplitude along the operator at one zero-offset sample.

    x [N, NT] aperture traces, dm [N] = m_i - m0, h [N] offsets, t0 = it0 dt.
    """
    x = np.asarray(x, np.float64)
    N = x.shape[0]
    if N == 0:
        return 0.0
    T = traveltime_sq(op, theta, t0, dm, h)
    a0 = window_amplitudes(x, T, dt, 0)[:, 0]
    return float(np.sum(a0) / N)


def stack_many(traces, mid, off, prob, theta, domains=None):
    """out[d] for theta [n_dom, D] (or [len(domains), D])."""
    theta = np.asarray(theta)
    doms = range(theta.shape[0]) if domains is None else domains
    out = np.zeros(theta.shape[0])
    for r, d in enumerate(doms):
        x, dt, dm, h, t0 = domain_data(traces, mid, off, prob, d)
        out[r] = stack(x, dt, dm, h, t0, prob.op, theta[r])
    return out
