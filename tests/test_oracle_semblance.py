"""Pins of the FP64 semblance oracle against closed forms and hand-worked cases.

Each check is independent of the oracle's own code path: hand-derived
values (tests/golden/semblance_worked.txt), events constructed here so that
every windowed amplitude is known exactly, Cauchy-Schwarz bounds, brute
force over parameter grids, and finite differences for the gradient.
"""
import math
import os

import numpy as np
import pytest

from oracle import semblance as osm

CMP, CRS, FOCRS = osm.CMP, osm.CRS, osm.FOCRS


def load_worked(path):
    cases, cur = [], None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "case":
            cur = dict(name=vals[0], traces=[], h0=0.0)
            cases.append(cur)
        elif key == "op":
            cur["op"] = {"CMP": CMP, "CRS": CRS, "FOCRS": FOCRS}[vals[0]]
        elif key in ("dt", "m0", "h0", "expect", "stack"):
            cur[key] = float(vals[0])
        elif key in ("w", "it0"):
            cur[key] = int(vals[0])
        elif key == "theta":
            cur["theta"] = [float(v) for v in vals]
        elif key == "trace":
            cur["traces"].append([float(v) for v in vals])
    return cases


def test_hand_worked_cases(golden_dir):
    cases = load_worked(os.path.join(golden_dir, "semblance_worked.txt"))
    assert len(cases) >= 6
    for c in cases:
        m = np.array([t[0] for t in c["traces"]])
        h = np.array([t[1] for t in c["traces"]])
        ns = max(len(t) - 2 for t in c["traces"])
        x = np.zeros((len(m), ns))
        for i, t in enumerate(c["traces"]):
            x[i, :len(t) - 2] = t[2:]
        if c["op"] == FOCRS:
            h = h - c["h0"]
        S = osm.semblance(x, c["dt"], m - c["m0"], h, c["it0"] * c["dt"], c["op"], c["theta"],
                          c["w"])
        assert S == pytest.approx(c["expect"], abs=1e-14), c["name"]


def _ramp_event(T, dt, ns, w, slope=0.37, base=1.0):
    """Traces x_i[n] = g(n dt - t_i) with g linear on |tau| <= (w+2) dt, zero
    elsewhere: linear interpolation is exact there, so every windowed
    amplitude is a_ik = g(k dt) whatever the fractional position."""
    t = np.sqrt(T)
    n = np.arange(ns)[None, :]
    tau = n * dt - t[:, None]
    g = base + slope * tau / dt
    return np.where(np.abs(tau) <= (w + 2) * dt, g, 0.0)


@pytest.mark.parametrize("op", [CMP, CRS])
def test_event_on_operator_gives_one(op):
    rng = np.random.default_rng(1)
    dt, ns, w = 0.004, 600, 5
    for _ in range(20):
        N = int(rng.integers(2, 60))
        dm = rng.uniform(-125, 125, N) if op == CRS else np.zeros(N)
        h = rng.uniform(0, 2350, N)
        it0 = int(rng.integers(50, 300))
        t0 = it0 * dt
        if op == CMP:
            theta = [rng.uniform(1 / 4500 ** 2, 1 / 1400 ** 2)]
            T = t0 * t0 + theta[0] * h * h
        else:
            theta = [rng.uniform(-4e-4, 4e-4), rng.uniform(-1e-7, 1e-7),
                     rng.uniform(1 / 4500 ** 2, 1 / 1400 ** 2)]
            T = (t0 + theta[0] * dm) ** 2 + theta[1] * dm * dm + theta[2] * h * h
        x = _ramp_event(T, dt, ns, w)
        S = osm.semblance(x, dt, dm, h, t0, op, theta, w)
        assert S == pytest.approx(1.0, abs=1e-12)
        # a perturbed parameter misaligns the event: S drops below 1
        bad = list(theta)
        bad[-1] *= 1.3
        if op == CRS:
            bad[0] = -theta[0] if abs(theta[0]) > 1e-4 else theta[0] + 3e-4
        assert osm.semblance(x, dt, dm, h, t0, op, bad, w) < 1.0 - 1e-6


def test_dip_sign_convention():
    """dm = m - m0: an event dipping with +A is flat only for +A."""
    dt, ns, w = 0.004, 400, 5
    dm = np.linspace(-100, 100, 17)
    h = np.zeros_like(dm)
    t0 = 100 * dt
    A = 3e-4
    T = (t0 + A * dm) ** 2
    x = _ramp_event(T, dt, ns, w)
    assert osm.semblance(x, dt, dm, h, t0, CRS, [A, 0.0, 0.0], w) == pytest.approx(1.0)
    assert osm.semblance(x, dt, dm, h, t0, CRS, [-A, 0.0, 0.0], w) < 0.9


def test_integer_sample_ricker_pythagorean():
    """t = 5 s dt for t0 = 3 s dt, C h^2 = (4 s dt)^2: every trace's window
    starts on a sample (f = 0) and holds the same Ricker samples -> S = 1."""
    dt, w = 0.004, 5
    ns = 400
    Cs = 1.0 / 2000.0 ** 2
    scales = [10, 14, 20, 26]
    t0 = 3 * 10 * dt
    x, h = [], []
    for s in scales:
        # T = (3*10 dt)^2 + C h^2 must equal (5 s' dt)^2 with integer samples:
        # choose h so that C h^2 = (k dt)^2 - t0^2 with k integer
        k = int(round(math.sqrt(t0 * t0 + Cs * (s * 40.0) ** 2) / dt))
        hh = math.sqrt(((k * dt) ** 2 - t0 * t0) / Cs)
        h.append(hh)
        n = np.arange(ns)
        tau = (n - k) * dt
        a = (math.pi * 25 * tau) ** 2
        x.append((1 - 2 * a) * np.exp(-a))
    x = np.array(x)
    h = np.array(h)
    S = osm.semblance(x, dt, np.zeros(len(h)), h, t0, CMP, [Cs], w)
    assert S == pytest.approx(1.0, abs=1e-9)


def test_single_trace_is_one():
    rng = np.random.default_rng(2)
    for _ in range(50):
        x = rng.standard_normal((1, 800))  # 3.2 s: the window stays on the record
        S = osm.semblance(x, 0.004, [0.0], [rng.uniform(0, 2000)], 0.2, CMP,
                          [rng.uniform(1e-8, 5e-7)], 5)
        assert S == pytest.approx(1.0, abs=1e-12)


def test_orthogonal_windows_give_one_over_n():
    """Trace i non-zero only at window position k = i: a_ik = c_i delta_ik,
    so s_k = c_k and S = sum c^2 / (N sum c^2) = 1/N."""
    w, dt = 5, 1.0
    for N in range(2, 2 * w + 2):
        x = np.zeros((N, 40))
        c = np.arange(1, N + 1, dtype=float)
        it0 = 20
        for i in range(N):
            x[i, it0 - w + i] = c[i]
        S = osm.semblance(x, dt, np.zeros(N), np.zeros(N), it0 * dt, CMP, [0.3], w)
        assert S == pytest.approx(1.0 / N, abs=1e-14)


def test_zero_window_is_zero():
    x = np.zeros((5, 100))
    assert osm.semblance(x, 0.004, np.zeros(5), np.arange(5) * 50.0, 0.1, CMP, [1e-7], 5) == 0.0
    # window entirely below the record: zero as well
    x = np.ones((3, 50))
    assert osm.semblance(x, 0.004, np.zeros(3), np.zeros(3), 0.4, CMP, [0.0], 5) == 0.0


def test_range_zero_one_random():
    rng = np.random.default_rng(3)
    for _ in range(200):
        N = int(rng.integers(1, 40))
        x = rng.standard_normal((N, 300))
        th = [rng.uniform(-6e-4, 6e-4), rng.uniform(-1.5e-7, 1.5e-7), rng.uniform(4e-8, 5e-7)]
        S = osm.semblance(x, 0.004, rng.uniform(-125, 125, N), rng.uniform(0, 2350, N),
                          rng.uniform(0, 1.2), CRS, th, 5)
        assert -1e-15 <= S <= 1.0 + 1e-12


def test_integer_u_is_plain_indexing():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 50))
    dt = 0.5
    u = np.array([7.0, 20.0, 33.0])
    T = (u * dt) ** 2
    a = osm.window_amplitudes(x, T, dt, 3)
    for i in range(3):
        j = int(u[i])
        np.testing.assert_array_equal(a[i], x[i, j - 3:j + 4])


def test_linear_interpolation_midpoint():
    x = np.array([[0.0, 2.0, 4.0, 10.0, 20.0, 0.0, 0.0]])
    a = osm.window_amplitudes(x, np.array([(2.25) ** 2]), 1.0, 1)
    # u = 2.25: samples (1,2),(2,3),(3,4) weighted 0.75 / 0.25
    np.testing.assert_allclose(a[0], [2.5, 5.5, 12.5], rtol=0, atol=1e-15)


def test_crs_reduces_to_cmp():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((30, 400))
    h = rng.uniform(0, 2350, 30)
    dm = rng.uniform(-100, 100, 30)
    for _ in range(20):
        C = rng.uniform(4e-8, 5e-7)
        t0 = rng.uniform(0, 1.5)
        s_cmp = osm.semblance(x, 0.004, np.zeros(30), h, t0, CMP, [C], 5)
        s_crs = osm.semblance(x, 0.004, np.zeros(30), h, t0, CRS, [0.0, 0.0, C], 5)
        s_crs_dm = osm.semblance(x, 0.004, dm, h, t0, CRS, [0.0, 0.0, C], 5)
        assert s_cmp == s_crs
        assert s_cmp == s_crs_dm  # A = B = 0: midpoint offsets play no role


def test_bruteforce_grid_recovers_cmp():
    """Tiny noise-free CMP gather, one Ricker event: grid argmax at the truth."""
    dt, ns, w = 0.004, 300, 5
    h = 50.0 * np.arange(24)
    t0e, v = 0.6, 2200.0
    C = 1.0 / v ** 2
    t = np.sqrt(t0e ** 2 + C * h * h)
    tau = np.arange(ns)[None, :] * dt - t[:, None]
    a = (math.pi * 25 * tau) ** 2
    x = (1 - 2 * a) * np.exp(-a)
    it0 = int(round(t0e / dt))
    vs = np.arange(1500.0, 4000.0, 10.0)
    S = [osm.semblance(x, dt, np.zeros(24), h, it0 * dt, CMP, [1 / vv ** 2], w) for vv in vs]
    assert abs(vs[int(np.argmax(S))] - v) <= 10.0
    assert max(S) > 0.99


def test_bruteforce_grid_recovers_crs():
    """Tiny noise-free 3-D (A, B, C) grid search on a 5-CMP gather."""
    dt, ns, w = 0.004, 300, 5
    mids = np.repeat(12.5 * np.arange(-2, 3), 12)
    h = np.tile(100.0 * np.arange(12), 5)
    A0, B0, C0, t0e = 2e-4, 4e-8, 1.0 / 2500 ** 2, 0.48
    T = (t0e + A0 * mids) ** 2 + B0 * mids ** 2 + C0 * h * h
    t = np.sqrt(T)
    tau = np.arange(ns)[None, :] * dt - t[:, None]
    a = (math.pi * 25 * tau) ** 2
    x = (1 - 2 * a) * np.exp(-a)
    it0 = int(round(t0e / dt))
    best, arg = -1, None
    for A in np.linspace(-4e-4, 4e-4, 9):
        for B in np.linspace(-1e-7, 1e-7, 5):
            for v in np.arange(1500.0, 4000.0, 100.0):
                S = osm.semblance(x, dt, mids, h, it0 * dt, CRS, [A, B, 1 / v ** 2], w)
                if S > best:
                    best, arg = S, (A, B, v)
    assert arg[0] == pytest.approx(A0, abs=1e-5)
    assert abs(arg[2] - 2500.0) <= 100.0
    assert best > 0.95


# --------------------------------------------------------------------------
# gradient
# --------------------------------------------------------------------------

def _fd_ok(x, dt, dm, h, t0, op, th, w, d, step):
    """True when a +-step in theta_d moves no trace across a sample (kink)."""
    for sgn in (-1.0, 0.0, 1.0):
        p = np.array(th, float)
        p[d] += sgn * step
        T = osm.traveltime_sq(op, p, t0, dm, h)
        if np.any(np.abs(T) < 1e-12):
            return False
        if sgn == -1.0:
            jm = np.floor(np.sqrt(np.maximum(T, 0)) / dt)
            negm = T < 0
        elif sgn == 1.0:
            jp = np.floor(np.sqrt(np.maximum(T, 0)) / dt)
            negp = T < 0
    return bool(np.all(jm == jp) and np.all(negm == negp))


@pytest.mark.parametrize("op", [CMP, CRS])
def test_gradient_matches_central_differences(op):
    rng = np.random.default_rng(6)
    dt, w = 0.004, 5
    lo = np.array([-6e-4, -1.5e-7, 1 / 4800 ** 2]) if op == CRS else np.array([1 / 4500 ** 2])
    hi = np.array([6e-4, 1.5e-7, 1 / 1400 ** 2]) if op == CRS else np.array([1 / 1400 ** 2])
    checked = 0
    for _ in range(60):
        N = int(rng.integers(5, 30))
        x = rng.standard_normal((N, 400))
        dm = rng.uniform(-125, 125, N) if op == CRS else np.zeros(N)
        h = rng.uniform(0, 2350, N)
        t0 = rng.uniform(0.1, 1.0)
        th = lo + rng.uniform(0, 1, lo.size) * (hi - lo)
        S, g = osm.semblance_grad(x, dt, dm, h, t0, op, th, w)
        assert S == pytest.approx(osm.semblance(x, dt, dm, h, t0, op, th, w), abs=1e-14)
        for d in range(lo.size):
            step = 1e-6 * max(abs(th[d]), hi[d] - lo[d])
            if not _fd_ok(x, dt, dm, h, t0, op, th, w, d, step):
                continue
            p, m = np.array(th), np.array(th)
            p[d] += step
            m[d] -= step
            fd = (osm.semblance(x, dt, dm, h, t0, op, p, w)
                  - osm.semblance(x, dt, dm, h, t0, op, m, w)) / (2 * step)
            scale = max(abs(fd), abs(g[d]), 1e-3 / (hi[d] - lo[d]))
            assert abs(fd - g[d]) <= 1e-5 * scale, (op, d, fd, g[d])
            checked += 1
    assert checked > 50


def test_gradient_flat_directions():
    """All traces at the reference midpoint (dm = 0): A and B drop out."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((20, 300))
    h = rng.uniform(0, 2000, 20)
    S, g = osm.semblance_grad(x, 0.004, np.zeros(20), h, 0.5, CRS, [2e-4, 5e-8, 2e-7], 5)
    assert g[0] == 0.0 and g[1] == 0.0
    S2, g2 = osm.semblance_grad(x, 0.004, np.zeros(20), h, 0.5, CMP, [2e-7], 5)
    assert S == pytest.approx(S2, abs=1e-15)
    assert g[2] == pytest.approx(g2[0], rel=1e-12)


def test_gradient_zero_at_exact_maximum():
    """A constant-amplitude event laid on the operator: S = 1 (the global
    maximum) and every windowed slope x[j+k+1] - x[j+k] is zero, so the
    analytic gradient vanishes."""
    dt, ns, w = 0.004, 400, 5
    h = 50.0 * np.arange(30)
    t0 = 100 * dt
    C = 1.0 / 2500 ** 2
    T = t0 * t0 + C * h * h
    x = _ramp_event(T, dt, ns, w, slope=0.0)  # constant amplitude event
    S, g = osm.semblance_grad(x, dt, np.zeros(30), h, t0, CMP, [C], w)
    assert S == pytest.approx(1.0)
    assert g[0] == pytest.approx(0.0, abs=1e-6 / C)


def test_gradient_at_zero_traveltime():
    """At t0 = 0 a zero-offset trace at the reference midpoint has T = 0 for
    every parameter vector: its amplitudes do not move, so it adds nothing to
    the gradient (and no 0/0), while the other traces do. The gradient stays
    finite and matches central differences."""
    rng = np.random.default_rng(8)
    dt, w = 0.004, 3
    x = rng.standard_normal((12, 200))
    dm = np.concatenate([[0.0], rng.uniform(-100, 100, 11)])
    h = np.concatenate([[0.0], rng.uniform(200, 2000, 11)])
    th = np.array([1e-4, 2e-8, 1 / 2500 ** 2])
    assert osm.traveltime_sq(CRS, th, 0.0, dm, h)[0] == 0.0
    S, g = osm.semblance_grad(x, dt, dm, h, 0.0, CRS, th, w)
    assert np.all(np.isfinite(g))
    for d, step in ((0, 1e-9), (2, 1e-12)):
        p, m = th.copy(), th.copy()
        p[d] += step
        m[d] -= step
        fd = (osm.semblance(x, dt, dm, h, 0.0, CRS, p, w)
              - osm.semblance(x, dt, dm, h, 0.0, CRS, m, w)) / (2 * step)
        assert fd == pytest.approx(g[d], rel=1e-4, abs=1e-6 * abs(g).max()), (d, fd, g[d])
