"""Pins of the stacked-output oracle (oracle.stack).

* Hand-worked values (tests/golden/semblance_worked.txt, "stack" lines,
  each derived from the centre stack sum printed with its case).
* A ramp event laid on the operator, scaled per trace: interpolation is exact
  there, so the stack is the mean scale times the ramp's value at the event.
* Integer positions (C = 0) reduce to plain indexing of the records.
* Linearity in the records, CRS with A = B = 0 equal to CMP, a trace with
  T < 0 adding zero but counting in N, positions past the record reading 0.
* Stacking N traces of independent noise divides its variance by N (the
  signal-to-noise gain the paper's Sec. 1 attributes to the operator).
"""
import os

import numpy as np
import pytest

from oracle import semblance as osm, stack as ost
from synth import configs
from test_oracle_semblance import load_worked

CMP, CRS = osm.CMP, osm.CRS


def test_hand_worked_stacks(golden_dir):
    cases = load_worked(os.path.join(golden_dir, "semblance_worked.txt"))
    assert sum("stack" in c for c in cases) >= 6
    for c in cases:
        m = np.array([t[0] for t in c["traces"]])
        h = np.array([t[1] for t in c["traces"]])
        ns = max(len(t) - 2 for t in c["traces"])
        x = np.zeros((len(m), ns))
        for i, t in enumerate(c["traces"]):
            x[i, :len(t) - 2] = t[2:]
        if c["op"] == osm.FOCRS:
            h = h - c["h0"]
        v = ost.stack(x, c["dt"], m - c["m0"], h, c["it0"] * c["dt"], c["op"], c["theta"])
        assert v == pytest.approx(c["stack"], abs=1e-14), c["name"]


@pytest.mark.parametrize("op", [CMP, CRS])
def test_scaled_ramp_event_on_operator(op):
    rng = np.random.default_rng(5)
    dt, ns = 0.004, 600
    for _ in range(20):
        N = int(rng.integers(1, 50))
        dm = rng.uniform(-125, 125, N) if op == CRS else np.zeros(N)
        h = rng.uniform(0, 2350, N)
        t0 = int(rng.integers(50, 300)) * dt
        if op == CMP:
            theta = [rng.uniform(1 / 4500 ** 2, 1 / 1400 ** 2)]
        else:
            theta = [rng.uniform(-4e-4, 4e-4), rng.uniform(-1e-7, 1e-7),
                     rng.uniform(1 / 4500 ** 2, 1 / 1400 ** 2)]
        T = osm.traveltime_sq(op, theta, t0, dm, h)
        tau = np.arange(ns)[None, :] * dt - np.sqrt(T)[:, None]
        ramp = np.where(np.abs(tau) <= 2 * dt, 0.8 + 0.3 * tau / dt, 0.0)
        alpha = rng.uniform(-1, 2, N)
        x = alpha[:, None] * ramp
        assert ost.stack(x, dt, dm, h, t0, op, theta) == pytest.approx(
            0.8 * alpha.mean(), abs=1e-12)


def test_integer_positions_are_plain_indexing():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(7, 40))
    for it0 in (0, 5, 39):
        v = ost.stack(x, 0.004, np.zeros(7), np.arange(7) * 50.0, it0 * 0.004, CMP, [0.0])
        assert v == pytest.approx(x[:, it0].mean(), abs=1e-14)


def test_linearity_crs_reduction_and_edges():
    rng = np.random.default_rng(7)
    N, ns, dt = 9, 200, 0.004
    x, y = rng.normal(size=(N, ns)), rng.normal(size=(N, ns))
    dm, h = rng.uniform(-100, 100, N), rng.uniform(0, 2000, N)
    th = [1e-4, 2e-8, 1 / 2500 ** 2]
    t0 = 0.3
    lhs = ost.stack(2.0 * x - 0.5 * y, dt, dm, h, t0, CRS, th)
    rhs = 2.0 * ost.stack(x, dt, dm, h, t0, CRS, th) - 0.5 * ost.stack(y, dt, dm, h, t0, CRS, th)
    assert lhs == pytest.approx(rhs, abs=1e-12)
    C = 1 / 3000 ** 2
    assert ost.stack(x, dt, dm, h, t0, CRS, [0.0, 0.0, C]) == pytest.approx(
        ost.stack(x, dt, dm, h, t0, CMP, [C]), abs=1e-15)
    # trace 0 has T < 0 (B dm^2 dominates): it adds 0, N stays 2
    x2 = np.ones((2, 50))
    v = ost.stack(x2, 0.01, np.array([10.0, 0.0]), np.zeros(2), 0.1, CRS, [0.0, -1.0, 0.0])
    assert v == pytest.approx(0.5, abs=1e-15)
    # every position past the record: 0; empty aperture: 0
    assert ost.stack(x2, 0.01, np.zeros(2), np.zeros(2), 0.1, CMP, [1.0]) == 1.0  # u = 10
    assert ost.stack(x2, 0.01, np.zeros(2), np.full(2, 100.0), 0.1, CMP, [1.0]) == 0.0
    assert ost.stack(np.zeros((0, 50)), 0.01, np.zeros(0), np.zeros(0), 0.1, CMP, [1.0]) == 0.0


def test_stack_divides_noise_variance_by_n():
    rng = np.random.default_rng(8)
    N, ns = 24, 20000
    x = rng.normal(size=(N, ns))
    st = np.array([ost.stack(x, 1.0, np.zeros(N), np.zeros(N), float(t), CMP, [0.0])
                   for t in range(0, ns, 4)])
    ratio = st.var() * N
    assert 0.9 < ratio < 1.1, ratio


def test_stack_many_matches_per_domain():
    wl = configs.crs_line(3, n_cmp=4, ns=60, n_events=2, ap_half=1, tau_max=0.2)
    prob = wl.problem
    rng = np.random.default_rng(9)
    lo, hi = np.array(configs.CRS_LO), np.array(configs.CRS_HI)
    th = lo + rng.uniform(0, 1, (prob.n_dom, 3)) * (hi - lo)
    many = ost.stack_many(wl.traces, wl.mid, wl.off, prob, th)
    for d in (0, 17, prob.n_dom - 1):
        x, dt, dm, h, t0 = osm.domain_data(wl.traces, wl.mid, wl.off, prob, d)
        assert many[d] == ost.stack(x, dt, dm, h, t0, prob.op, th[d])
