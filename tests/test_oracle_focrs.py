"""Pins of the FO-CRS operator in the oracle (op FOCRS, theta = Am, Ah, Bmm,
Bmh, Bhh on a common-offset section at central offset h0).

* Hand-worked value (the focrs case of tests/golden/semblance_worked.txt,
  covered by the fixture tests).
* Reduction: with h0 = 0, Ah = 0, Bmh = 0, Bhh = C the operator is the CRS
  operator, bit for bit, and so is the semblance.
* Re-expansion identity: a synthetic event's traveltime surface re-expanded
  about (m0, h0) (synth.fo_recentre, the term-by-term match of two
  quadratics) gives, through the operator, the event's own t^2 at every
  (m, h): a dropped term, a wrong sign or a swapped slope breaks it.
* A ramp event laid on the operator gives S = 1; moving any one of the five
  parameters lowers S.
* Brute force on a tiny section finds the generating slopes (Am, Ah) on a
  grid with the curvatures fixed, and the generating curvature pair
  (Bmh, Bhh) with the slopes fixed.
* The analytic gradient matches central differences in all five directions.
"""
import numpy as np
import pytest

from oracle import semblance as osm
import synth
from synth import configs

FOCRS, CRS = osm.FOCRS, osm.CRS


def test_reduces_to_crs():
    rng = np.random.default_rng(0)
    for _ in range(50):
        dm, h = rng.uniform(-150, 150, 30), rng.uniform(0, 2350, 30)
        A, B, C = rng.uniform(-4e-4, 4e-4), rng.uniform(-1e-7, 1e-7), rng.uniform(5e-8, 4e-7)
        t0 = rng.uniform(0.2, 2.0)
        Tc = osm.traveltime_sq(CRS, [A, B, C], t0, dm, h)
        Tf = osm.traveltime_sq(FOCRS, [A, 0.0, B, 0.0, C], t0, dm, h)   # h0 = 0: dh = h
        np.testing.assert_array_equal(Tc, Tf)
    x = rng.normal(size=(30, 400))
    assert osm.semblance(x, 0.004, dm, h, 0.8, FOCRS, [A, 0, B, 0, C], 5) == \
        osm.semblance(x, 0.004, dm, h, 0.8, CRS, [A, B, C], 5)


def test_recentred_event_lies_on_the_operator():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(200):
        ev = [rng.uniform(0, 2500), rng.uniform(0.2, 5.5), rng.uniform(-4e-4, 4e-4),
              rng.uniform(-1e-7, 1e-7), 1 / rng.uniform(1500, 4500) ** 2, 1.0]
        m0, h0 = rng.uniform(0, 2500), rng.uniform(0, 2350)
        p = synth.gathers.fo_recentre(ev, m0, h0)
        if p is None:
            continue
        t0, th = p[0], p[1:]
        m = m0 + rng.uniform(-150, 150, 40)
        h = np.clip(h0 + rng.uniform(-1000, 1000, 40), 0, None)
        dme = m - ev[0]
        truth = (ev[1] + ev[2] * dme) ** 2 + ev[3] * dme ** 2 + ev[4] * h ** 2
        T = osm.traveltime_sq(FOCRS, th, t0, m - m0, h - h0)
        np.testing.assert_allclose(T, truth, rtol=1e-10, atol=1e-12)
        checked += 1
    assert checked > 150


def _ramp_section(theta, t0, dm, dh, dt, ns, w, slope=0.41):
    T = osm.traveltime_sq(FOCRS, theta, t0, dm, dh)
    t = np.sqrt(T)
    tau = np.arange(ns)[None, :] * dt - t[:, None]
    return np.where(np.abs(tau) <= (w + 2) * dt, 1.0 + slope * tau / dt, 0.0)


def test_ramp_event_on_operator_and_each_parameter_matters():
    rng = np.random.default_rng(2)
    dt, ns, w = 0.004, 700, 5
    for _ in range(10):
        N = 60
        dm, dh = rng.uniform(-100, 100, N), rng.uniform(-1000, 1000, N)
        t0 = int(rng.integers(150, 400)) * dt
        th = [rng.uniform(-4e-4, 4e-4), rng.uniform(0, 6e-4), rng.uniform(-1e-7, 2e-7),
              rng.uniform(-5e-7, 5e-7), rng.uniform(1e-8, 4e-7)]
        x = _ramp_section(th, t0, dm, dh, dt, ns, w)
        assert osm.semblance(x, dt, dm, dh, t0, FOCRS, th, w) == pytest.approx(1.0, abs=1e-12)
        steps = [3e-4, 3e-4, 4e-7, 8e-7, 2e-7]
        for k in range(5):
            bad = list(th)
            bad[k] += steps[k]
            assert osm.semblance(x, dt, dm, dh, t0, FOCRS, bad, w) < 1.0 - 1e-6, k


def test_brute_force_recovers_slopes_and_curvatures():
    rng = np.random.default_rng(3)
    dt, ns, w, N = 0.004, 500, 3, 80
    dm, dh = rng.uniform(-100, 100, N), rng.uniform(-1000, 1000, N)
    t0 = 1.0
    th = [2.5e-4, 4.0e-4, 1.0e-7, -2.0e-7, 2.0e-7]
    x = _ramp_section(th, t0, dm, dh, dt, ns, w)
    grid_m = np.linspace(-5e-4, 5e-4, 21)       # contains 2.5e-4
    grid_h = np.linspace(0.0, 8e-4, 21)         # contains 4e-4
    S = np.array([[osm.semblance(x, dt, dm, dh, t0, FOCRS, [a, b] + th[2:], w) for b in grid_h]
                  for a in grid_m])
    i, j = np.unravel_index(np.argmax(S), S.shape)
    assert grid_m[i] == pytest.approx(th[0]) and grid_h[j] == pytest.approx(th[1])
    grid_mh = np.linspace(-6e-7, 6e-7, 13)      # contains -2e-7
    grid_hh = np.linspace(0.0, 4e-7, 11)        # contains 2e-7
    S = np.array([[osm.semblance(x, dt, dm, dh, t0, FOCRS, th[:3] + [p, q], w) for q in grid_hh]
                  for p in grid_mh])
    i, j = np.unravel_index(np.argmax(S), S.shape)
    assert grid_mh[i] == pytest.approx(th[3]) and grid_hh[j] == pytest.approx(th[4])


def test_gradient_matches_central_differences():
    wl = configs.fo_panel(4, n_cmp=10, ns=300, n_events=3, tau_max=0.9)
    prob = wl.problem
    rng = np.random.default_rng(4)
    lo, hi = np.array(configs.FO_LO), np.array(configs.FO_HI)
    checked = 0
    for d in rng.choice(prob.n_dom, 40, replace=False):
        x, dt, dm, dh, t0 = osm.domain_data(wl.traces, wl.mid, wl.off, prob, d)
        th = lo + rng.uniform(0, 1, 5) * (hi - lo)
        S, g = osm.semblance_grad(x, dt, dm, dh, t0, FOCRS, th, 5)
        if S == 0.0:
            continue
        for k in range(5):
            hk = 1e-6 * (hi[k] - lo[k])
            tp, tm = th.copy(), th.copy()
            tp[k] += hk
            tm[k] -= hk
            # skip kinks: a trace crossing a sample between the two points
            up = np.sqrt(np.maximum(osm.traveltime_sq(FOCRS, tp, t0, dm, dh), 0)) / dt
            um = np.sqrt(np.maximum(osm.traveltime_sq(FOCRS, tm, t0, dm, dh), 0)) / dt
            if np.any(np.floor(up) != np.floor(um)):
                continue
            fd = (osm.semblance(x, dt, dm, dh, t0, FOCRS, tp, 5) -
                  osm.semblance(x, dt, dm, dh, t0, FOCRS, tm, 5)) / (2 * hk)
            assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 / (hi[k] - lo[k])), (d, k)
            checked += 1
    assert checked >= 60


def test_section_geometry_at_recentred_parameters():
    """On a noise-free section the event-centred domains reach S > 0.9 at the
    re-expanded parameters (which needs dh = h - h0 in the domain geometry)
    and far less at the parameters re-expanded about the wrong offset."""
    wl = configs.fo_panel(5, n_cmp=16, ns=400, n_events=2, snr=0.0, tau_max=1.0)
    prob, line = wl.problem, wl.line
    tried = 0
    for ev in line.events:
        c = int(np.argmin(np.abs(line.cmp_x - ev[0])))
        if not 3 <= c < line.n_cmp - 3:
            continue
        p = synth.gathers.fo_recentre(ev, line.cmp_x[c], 1000.0)
        q = synth.gathers.fo_recentre(ev, line.cmp_x[c], 0.0)
        it0 = int(round(p[0] / line.dt))
        if not 10 <= it0 < line.ns - 10:
            continue
        d = c * prob.n_t0 + it0
        S = osm.semblance_many(wl.traces, wl.mid, wl.off, prob, np.array([[p[1:], q[1:]]]),
                               domains=[d])[0]
        assert S[0] > 0.9 and S[1] < 0.5 * S[0], (S, ev)
        tried += 1
    assert tried >= 1
