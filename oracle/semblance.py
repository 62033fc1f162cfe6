"""FP64 semblance of a traveltime operator and its gradient (TEST INFRASTRUCTURE).

The paper names the objective (Semblance, Neidell & Taner 1971, Sec. 1) and
the operators (CMP, Mayne 1962; CRS, Jaeger 2001; Sec. 1) but prints no
formula for either; Sec. 2 (eq. order) states that one semblance call costs
W_l x T_a (window length x aperture traces) and Sec. 2.2 (eq. S) that it
maps into [0, 1]. The readings adopted here:

* Traveltime, squared, at a trace of midpoint m and full offset h for the
  zero-offset sample (m0, t0), with dm = m - m0:
    CMP  (theta = C):        T = t0^2 + C h^2
    CRS  (theta = A, B, C):  T = (t0 + A dm)^2 + B dm^2 + C h^2
  t = sqrt(T); where T < 0 the trace contributes zeros (it still counts in N).
* FO-CRS (Sec. 1: two slopes and three wavefront curvatures; the hyperbolic
  finite-offset CRS operator of the cited Zhang et al. 2001), for the sample
  t0 of a common-offset section at central full offset h0, with
  dh = h - h0 (the ``h`` argument of the functions below is then dh):
    FO-CRS (theta = Am, Ah, Bmm, Bmh, Bhh):
      T = (t0 + Am dm + Ah dh)^2 + Bmm dm^2 + Bmh dm dh + Bhh dh^2,
  the second-order (hyperbolic) expansion of t^2 in the midpoint and offset
  displacements; its physical parameters (emergence angles, curvatures) are
  absorbed into the five coefficients, as the CRS constants are into A, B, C.
  With h0 = 0, Ah = 0, Bmh = 0 and Bhh = C it is the CRS operator.
* Window: the 2w+1 samples at t + k dt, k = -w..w, read by linear
  interpolation: with u = t/dt, j = floor(u), f = u - j,
    a_k = (1 - f) x[j + k] + f x[j + k + 1],   x[n] = 0 outside [0, NT-1].
* Semblance over the N aperture traces i:
    s_k = sum_i a_ik,  E = sum_i sum_k a_ik^2,  S = sum_k s_k^2 / (N E),
  and S = 0 where E = 0. By Cauchy-Schwarz 0 <= S <= 1 (Sec. 2.2, eq. S).

Everything is float64; the record may be stored in any float type.
"""
from __future__ import annotations

import numpy as np

CMP, CRS, FOCRS = 0, 1, 2


def traveltime_sq(op: int, theta, t0, dm, h):
    """Squared traveltime T (s^2) of the operator (readings in module doc)."""
    h = np.asarray(h, np.float64)
    dm = np.asarray(dm, np.float64)
    if op == CMP:
        (C,) = (float(v) for v in theta)
        return t0 * t0 + C * h * h
    if op == FOCRS:
        Am, Ah, Bmm, Bmh, Bhh = (float(v) for v in theta)
        dh = h
        return (t0 + Am * dm + Ah * dh) ** 2 + Bmm * dm * dm + Bmh * dm * dh + Bhh * dh * dh
    A, B, C = (float(v) for v in theta)
    return (t0 + A * dm) ** 2 + B * dm * dm + C * h * h


def record_sample(x: np.ndarray, n: np.ndarray) -> np.ndarray:
    """x[i, n] for integer sample indices n [..., N, K] of trace i (axis -2),
    zero outside the record [0, NT-1]; x is [N, NT]."""
    NT = x.shape[1]
    inside = (n >= 0) & (n < NT)
    rows = np.arange(x.shape[0])[:, None]
    return np.where(inside, x[rows, np.clip(n, 0, NT - 1)], 0.0)


def window_amplitudes(x: np.ndarray, T: np.ndarray, dt: float, w: int) -> np.ndarray:
    """a[..., i, k] (k = -w..w) for traces x [N, NT] and squared times T [..., N]."""
    T = np.asarray(T, np.float64)
    ok = T >= 0.0
    u = np.sqrt(np.where(ok, T, 0.0)) / dt
    j = np.floor(u)
    f = (u - j)[..., None]
    k = np.arange(-w, w + 1)
    n0 = j.astype(np.int64)[..., None] + k
    a = (1.0 - f) * record_sample(x, n0) + f * record_sample(x, n0 + 1)
    return np.where(ok[..., None], a, 0.0)


def semblance_from_amplitudes(a: np.ndarray):
    """S = sum_k (sum_i a_ik)^2 / (N sum_ik a_ik^2) over the last two axes
    (i, k) of a; 0 where the energy is 0."""
    N = a.shape[-2]
    E = np.sum(a * a, axis=(-2, -1))
    s = np.sum(a, axis=-2)
    Q = np.sum(s * s, axis=-1)
    safe = np.where(E > 0.0, E, 1.0)
    S = np.where((E > 0.0) & (N > 0), Q / (max(N, 1) * safe), 0.0)
    return float(S) if S.ndim == 0 else S


def traveltime_sq_population(op: int, thetas, t0, dm, h):
    """T [P, N] for parameter vectors thetas [P, D]."""
    thetas = np.asarray(thetas, np.float64)
    return np.stack([traveltime_sq(op, th, t0, dm, h) for th in thetas])


def semblance(x, dt, dm, h, t0, op, theta, w):
    """S at one zero-offset sample for one parameter vector.

    x [N, NT] aperture traces, dm [N] = m_i - m0, h [N] offsets, t0 = it0 dt.
    """
    x = np.asarray(x, np.float64)
    T = traveltime_sq(op, theta, t0, dm, h)
    return semblance_from_amplitudes(window_amplitudes(x, T, dt, w))


def semblance_grad(x, dt, dm, h, t0, op, theta, w):
    """(S, dS/dtheta) at one point, by the chain rule through the window.

    With Q = sum_k s_k^2, dS/da_ik = 2 s_k / (N E) - 2 S a_ik / E; inside an
    interpolation cell da_ik/du_i = x[j+k+1] - x[j+k]; du/dtheta =
    (dT/dtheta) / (2 t dt) with dT/dA = 2 (t0 + A dm) dm, dT/dB = dm^2,
    dT/dC = h^2 (CMP: only dT/dC); FO-CRS, with q = t0 + Am dm + Ah dh:
    dT/dAm = 2 q dm, dT/dAh = 2 q dh, dT/dBmm = dm^2, dT/dBmh = dm dh,
    dT/dBhh = dh^2. Traces with T < 0, or t = 0, add nothing; E = 0 gives
    S = 0 and a zero gradient.
    """
    x = np.asarray(x, np.float64)
    dm = np.asarray(dm, np.float64)
    h = np.asarray(h, np.float64)
    D = {CMP: 1, CRS: 3, FOCRS: 5}[op]
    T = traveltime_sq(op, theta, t0, dm, h)
    a = window_amplitudes(x, T, dt, w)
    N = a.shape[0]
    E = float(np.sum(a * a))
    if E == 0.0 or N == 0:
        return 0.0, np.zeros(D)
    s = np.sum(a, axis=0)
    S = float(np.sum(s * s) / (N * E))
    dS_da = 2.0 * s[None, :] / (N * E) - 2.0 * S * a / E
    ok = T > 0.0
    t = np.sqrt(np.where(ok, T, 1.0))
    u = t / dt
    j = np.floor(u).astype(np.int64)
    k = np.arange(-w, w + 1)[None, :]
    slope = record_sample(x, j[:, None] + k + 1) - record_sample(x, j[:, None] + k)
    dS_du = np.where(ok, np.sum(dS_da * slope, axis=1), 0.0)
    if op == CMP:
        dT = [h * h]
    elif op == FOCRS:
        q = t0 + float(theta[0]) * dm + float(theta[1]) * h
        dT = [2.0 * q * dm, 2.0 * q * h, dm * dm, dm * h, h * h]
    else:
        A = float(theta[0])
        dT = [2.0 * (t0 + A * dm) * dm, dm * dm, h * h]
    g = np.array([np.sum(dS_du * dTd / (2.0 * t * dt)) for dTd in dT])
    return S, g


# --------------------------------------------------------------------------
# Many domains x many individuals (problem given as plain arrays)
# --------------------------------------------------------------------------

def _domain_geometry(traces, mid, off, prob, d):
    g = int(prob.dom_group[d])
    idx = prob.ap_idx[prob.ap_ptr[g]:prob.ap_ptr[g + 1]]
    dt = float(prob.group_dt[g])
    x = np.asarray(traces[idx], np.float64)
    dm = np.asarray(mid[idx], np.float64) - float(prob.group_m0[g])
    h = np.asarray(off[idx], np.float64)
    if prob.op == FOCRS:   # offset displacement from the section's central offset
        h = h - float(prob.group_h0[g])
    t0 = float(prob.dom_it0[d]) * dt
    return x, dt, dm, h, t0


def semblance_many(traces, mid, off, prob, theta, domains=None):
    """S[d, p] for theta [n_dom, P, D] (or [len(domains), P, D]).

    ``prob`` is any object with the attributes op, half_window, group_m0,
    group_dt, ap_ptr, ap_idx, dom_it0, dom_group (and group_h0 for FO-CRS).
    """
    theta = np.asarray(theta)
    doms = range(theta.shape[0]) if domains is None else domains
    out = np.zeros(theta.shape[:2])
    for r, d in enumerate(doms):
        x, dt, dm, h, t0 = _domain_geometry(traces, mid, off, prob, d)
        T = traveltime_sq_population(prob.op, theta[r], t0, dm, h)
        out[r] = semblance_from_amplitudes(window_amplitudes(x, T, dt, prob.half_window))
    return out


def semblance_grad_many(traces, mid, off, prob, theta, domains=None):
    """(S[d, p], dS[d, p, D]) for theta [n_dom, P, D]."""
    theta = np.asarray(theta)
    doms = range(theta.shape[0]) if domains is None else domains
    S = np.zeros(theta.shape[:2])
    G = np.zeros(theta.shape)
    for r, d in enumerate(doms):
        x, dt, dm, h, t0 = _domain_geometry(traces, mid, off, prob, d)
        for p in range(theta.shape[1]):
            S[r, p], G[r, p] = semblance_grad(x, dt, dm, h, t0, prob.op, theta[r, p],
                                              prob.half_window)
    return S, G


def domain_data(traces, mid, off, prob, d):
    """Aperture traces and geometry of domain d: (x, dt, dm, h, t0); for
    FO-CRS h is the offset displacement dh = h - h0."""
    return _domain_geometry(traces, mid, off, prob, d)
