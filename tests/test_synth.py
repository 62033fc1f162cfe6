"""Pins of the seeded input generator (synth/): the wavelet, the event
surfaces, the noise level, the layouts, and the closed-form recentring that
serves as ground truth for recovered parameters."""
import math

import numpy as np
import pytest

import synth
from synth import gathers

OFF = 50.0 * np.arange(48)


def _line(snr, seed=4, n_events=1, **kw):
    args = dict(n_cmp=6, dcmp=12.5, offsets=OFF, ns=400, dt=0.004, n_events=n_events,
                tau_range=(0.4, 1.0), A_range=(-4e-4, 4e-4), B_range=(-1e-7, 1e-7),
                v_range=(1800.0, 3500.0), snr=snr, seed=seed)
    args.update(kw)
    return gathers.make_line(**args)


def test_ricker_shape():
    f = 25.0
    assert gathers.ricker(np.array([0.0]), f)[0] == 1.0
    z = 1.0 / (math.pi * f * math.sqrt(2.0))          # zero crossings
    assert np.allclose(gathers.ricker(np.array([-z, z]), f), 0.0, atol=1e-15)
    tm = math.sqrt(1.5) / (math.pi * f)                # side lobes: -2 e^(-3/2)
    assert np.allclose(gathers.ricker(np.array([-tm, tm]), f), -2.0 * math.exp(-1.5))
    tau = np.linspace(-0.05, 0.05, 101)
    assert np.allclose(gathers.ricker(tau, f), gathers.ricker(-tau, f))


def test_event_peaks_on_its_traveltime_surface():
    """Noise free, one event: on every trace where it arrives the largest
    amplitude lies within one sample of t_e(m, h), with the event's sign."""
    line = _line(snr=0)
    m_e, tau, A, B, C, amp = line.events[0]
    dm = line.mid.astype(np.float64) - m_e
    T = (tau + A * dm) ** 2 + B * dm * dm + C * line.off.astype(np.float64) ** 2
    t = np.sqrt(T)
    for i in range(line.n_tr):
        n_pk = int(np.argmax(np.abs(line.traces[i])))
        if t[i] / line.dt >= line.ns - 2:
            continue
        assert abs(n_pk - t[i] / line.dt) <= 1.0, i
        assert np.sign(line.traces[i, n_pk]) == np.sign(amp)
        assert abs(line.traces[i, n_pk]) <= abs(amp) + 1e-6


def test_noise_level_is_peak_over_snr():
    clean = _line(snr=0, seed=9, n_events=3)
    noisy = _line(snr=4.0, seed=9, n_events=3)
    np.testing.assert_array_equal(clean.events, noisy.events)
    resid = (noisy.traces - clean.traces).astype(np.float64)
    sigma = float(np.max(np.abs(clean.traces))) / 4.0
    assert resid.std() == pytest.approx(sigma, rel=0.01)
    assert abs(resid.mean()) < 0.01 * sigma


def test_line_layout_and_apertures():
    line = _line(snr=0, n_cmp=7)
    assert np.array_equal(line.mid[:48], np.full(48, line.cmp_x[0], np.float32))
    assert np.array_equal(line.off[48:96], OFF.astype(np.float32))
    prob = synth.line_problem(line, half_window=5, ap_half=2, cmps=[0, 3, 6],
                              t0_range=(10, 14))
    assert (prob.n_m0, prob.n_t0, prob.n_dom) == (3, 4, 12)
    # m0-major domains, the aperture +-2 CMPs clipped at the line ends
    assert list(prob.dom_group) == [0] * 4 + [1] * 4 + [2] * 4
    assert list(prob.dom_it0[:4]) == [10, 11, 12, 13]
    cm = [sorted(set((line.mid[prob.aperture(g)] / 12.5).round().astype(int)))
          for g in range(3)]
    assert cm == [[0, 1, 2], [1, 2, 3, 4, 5], [4, 5, 6]]


@pytest.mark.parametrize("seed", range(5))
def test_crs_recentring_reproduces_the_event_surface(seed):
    """The recentred (t0, A', B', C) about any m0 give back the event's own
    squared traveltime at every (m, h): an identity in m, so at any
    displacement from m0."""
    rng = np.random.default_rng(seed)
    ev = np.array([100.0, rng.uniform(0.3, 1.5), rng.uniform(-4e-4, 4e-4),
                   rng.uniform(-1e-7, 1e-7), 1 / rng.uniform(1500, 4000) ** 2, 1.0])
    m0 = 100.0 + rng.uniform(-150, 150)
    t0, Ap, Bp, Cp = gathers.crs_recentre(ev, m0)
    m = m0 + rng.uniform(-300, 300, 50)
    h = rng.uniform(0, 3000, 50)
    T_ev = (ev[1] + ev[2] * (m - ev[0])) ** 2 + ev[3] * (m - ev[0]) ** 2 + ev[4] * h * h
    T_op = (t0 + Ap * (m - m0)) ** 2 + Bp * (m - m0) ** 2 + Cp * h * h
    np.testing.assert_allclose(T_op, T_ev, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_fo_recentring_reproduces_the_event_surface(seed):
    rng = np.random.default_rng(10 + seed)
    ev = np.array([100.0, rng.uniform(0.3, 1.5), rng.uniform(-4e-4, 4e-4),
                   rng.uniform(-1e-7, 1e-7), 1 / rng.uniform(1500, 4000) ** 2, 1.0])
    m0, h0 = 100.0 + rng.uniform(-150, 150), rng.uniform(200, 2000)
    t0, Am, Ah, Bmm, Bmh, Bhh = gathers.fo_recentre(ev, m0, h0)
    dm = rng.uniform(-300, 300, 50)
    dh = rng.uniform(-h0, 1000, 50)
    m, h = m0 + dm, h0 + dh
    T_ev = (ev[1] + ev[2] * (m - ev[0])) ** 2 + ev[3] * (m - ev[0]) ** 2 + ev[4] * h * h
    T_op = (t0 + Am * dm + Ah * dh) ** 2 + Bmm * dm * dm + Bmh * dm * dh + Bhh * dh * dh
    np.testing.assert_allclose(T_op, T_ev, rtol=1e-12, atol=1e-14)


def test_recentring_absent_arrival():
    # an event whose zero-offset time squared is negative at m0 has no parameters there
    ev = np.array([0.0, 0.1, 0.0, -1e-6, 1e-7, 1.0])
    assert gathers.crs_recentre(ev, 500.0) is None
    assert gathers.fo_recentre(ev, 500.0, 0.0) is None
