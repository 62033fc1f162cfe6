"""The five workloads (and small variants of them) as seeded builders.

Each builder returns a ``Workload``: the line (or packed batch), the problem
(domains, groups, apertures) and the differential-evolution settings. The
paper's datasets are not available; these synthetic lines take their shapes
(trace and sample counts, offsets, window, aperture) from the workloads the
search is measured on. Sizes in the names are the full-size ones.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .gathers import (CMP, CRS, FOCRS, Line, Problem, make_line, cmp_problem, line_problem,
                      fo_problem, batched_problems)


@dataclasses.dataclass
class DEConfig:
    np: int
    ng: int
    F: float
    CR: float
    seed: int
    lo: tuple
    hi: tuple
    exch_every: int = 0
    polish_steps: int = 0
    polish_lr: float = 0.0
    adapt: int = 0           # 1: JADE adaptation of F, CR (initial mu = F, CR) + archive

    def as_arrays(self):
        return np.asarray(self.lo, np.float32), np.asarray(self.hi, np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    traces: np.ndarray
    mid: np.ndarray
    off: np.ndarray
    dt: float
    problem: Problem
    de: DEConfig
    storage: str = "f32"     # "f32" or "bf16"
    line: Line | None = None
    info: dict | None = None


OFF_48 = 50.0 * np.arange(48)        # 0 .. 2350 m
OFF_120 = 50.0 * np.arange(120)      # 0 .. 5950 m
C_BOUNDS_CMP = (1.0 / 4500.0 ** 2, 1.0 / 1400.0 ** 2)
CRS_LO = (-6e-4, -1.5e-7, 1.0 / 4800.0 ** 2)
CRS_HI = (6e-4, 1.5e-7, 1.0 / 1400.0 ** 2)
POLISH_LR = 2e-4
# FO-CRS (Am, Ah, Bmm, Bmh, Bhh) on a common-offset section at h0 <= 2350 m,
# from the recentring formulas over the crs_line generating ranges near the
# events (|Am| <~ |A|, 0 <= Ah = C h0 / t0 <= sqrt(C) <= 1/1400,
# Bmm = A^2 + B - Am^2, Bmh = -2 Am Ah, 0 <= Bhh = C - Ah^2 <= C), widened
FO_LO = (-6e-4, -1e-4, -3e-7, -1e-6, -2e-8)
FO_HI = (6e-4, 8e-4, 3e-7, 1e-6, 1.0 / 1400.0 ** 2 + 2e-8)


def cmp_search(seed: int = 0, *, ns: int = 500, n_events: int = 8, np_: int = 32,
               ng: int = 50, polish_steps: int = 0) -> Workload:
    """CMP search, plain FP32: one CMP gather of 48 traces (0-2350 m at 50 m),
    500 samples at 4 ms, 8 Ricker events with t0 in 0.2-1.9 s and C = 1/v^2,
    v in 1500-4000 m/s, SNR 5; window 11 samples; DE 32 x 50, F 0.5, CR 0.9."""
    line = make_line(n_cmp=1, dcmp=12.5, offsets=OFF_48, ns=ns, dt=0.004,
                     n_events=n_events, tau_range=(0.2, 1.9), A_range=None,
                     B_range=None, v_range=(1500.0, 4000.0), snr=5.0, seed=seed)
    prob = cmp_problem(line, half_window=5)
    de = DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=seed, lo=(C_BOUNDS_CMP[0],),
                  hi=(C_BOUNDS_CMP[1],), polish_steps=polish_steps, polish_lr=POLISH_LR)
    return Workload("cmp_1x48x500", line.traces, line.mid, line.off, line.dt, prob, de, line=line)


def crs_line(seed: int = 0, *, n_cmp: int = 200, ns: int = 1500, n_events: int = 20,
             ap_half: int = 10, np_: int = 64, ng: int = 100, exch_every: int = 10,
             polish_steps: int = 5, cmps=None, t0_range=None, snr: float = 3.0,
             tau_max: float | None = None) -> Workload:
    """CRS (A, B, C) search with neighbour exchange, FP32: 200 CMPs at 12.5 m,
    48 offsets, 1500 samples at 4 ms, 20 dipping events (A in +-4e-4 s/m,
    B in +-1e-7 s^2/m^2, v in 1500-4500 m/s), SNR 3, aperture +-10 CMPs,
    DE 64 x 100, exchange with the 4 adjacent domains every 10 generations,
    5 gradient-polish steps."""
    dt = 0.004
    tmax = (ns - 1) * dt
    line = make_line(n_cmp=n_cmp, dcmp=12.5, offsets=OFF_48, ns=ns, dt=dt, n_events=n_events,
                     tau_range=(0.2, tau_max if tau_max else 0.93 * tmax),
                     A_range=(-4e-4, 4e-4), B_range=(-1e-7, 1e-7),
                     v_range=(1500.0, 4500.0), snr=snr, seed=seed)
    prob = line_problem(line, half_window=5, ap_half=ap_half, cmps=cmps, t0_range=t0_range)
    de = DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=seed, lo=CRS_LO, hi=CRS_HI,
                  exch_every=exch_every, polish_steps=polish_steps, polish_lr=POLISH_LR)
    return Workload(f"crs_line_{n_cmp}x48x{ns}", line.traces, line.mid, line.off, dt, prob, de,
                    line=line)


def fo_panel(seed: int = 0, *, n_cmp: int = 200, ns: int = 1500, n_events: int = 20,
             h0: float = 1000.0, ap_half: int = 8, off_half: float = 1000.0, np_: int = 64,
             ng: int = 100, exch_every: int = 10, polish_steps: int = 0, cmps=None,
             t0_range=None, snr: float = 3.0, tau_max: float | None = None) -> Workload:
    """FO-CRS (Am, Ah, Bmm, Bmh, Bhh) search on the common-offset section at
    h0 = 1000 m of the CRS line's data (200 CMPs x 48 offsets x 1500 samples
    at 4 ms, 20 events, SNR 3): midpoint aperture +-8 CMPs (+-100 m), offset
    aperture +-1000 m (41 offsets), window 11, DE 64 x 100 with exchange."""
    dt = 0.004
    tmax = (ns - 1) * dt
    line = make_line(n_cmp=n_cmp, dcmp=12.5, offsets=OFF_48, ns=ns, dt=dt, n_events=n_events,
                     tau_range=(0.2, tau_max if tau_max else 0.93 * tmax),
                     A_range=(-4e-4, 4e-4), B_range=(-1e-7, 1e-7), v_range=(1500.0, 4500.0),
                     snr=snr, seed=seed)
    prob = fo_problem(line, half_window=5, h0=h0, ap_half=ap_half, off_half=off_half,
                      cmps=cmps, t0_range=t0_range)
    de = DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=seed, lo=FO_LO, hi=FO_HI,
                  exch_every=exch_every, polish_steps=polish_steps, polish_lr=POLISH_LR)
    return Workload(f"fo_{n_cmp}x48x{ns}_h{int(h0)}", line.traces, line.mid, line.off, dt, prob,
                    de, line=line)


def batched(seed: int = 0, *, n_prob: int = 4096, ntr_range=(16, 240), ns_range=(750, 3000),
            np_: int = 64, ng: int = 80, domains_per_problem=None) -> Workload:
    """Batched uneven gathers, FP32: 4096 independent CRS problems with
    16-240 traces and 750-3000 samples at 2 or 4 ms each; DE 64 x 80."""
    tr, mid, off, prob, info = batched_problems(
        n_prob=n_prob, ntr_range=ntr_range, ns_range=ns_range, dts=(0.002, 0.004), seed=seed,
        domains_per_problem=domains_per_problem)
    de = DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=seed, lo=CRS_LO, hi=CRS_HI)
    return Workload(f"batched_{n_prob}", tr, mid, off, 0.004, prob, de, info=info)


def large_line(seed: int = 0, *, n_cmp: int = 2000, ns: int = 2000, n_events: int = 60,
               ap_half: int = 25, np_: int = 96, ng: int = 120, cmps=None,
               t0_range=None) -> Workload:
    """Large line, BF16-stored traces: 2000 CMPs at 12.5 m, 120 offsets
    (0-5950 m), 2000 samples at 2 ms, 60 events, SNR 2, aperture +-25 CMPs,
    DE 96 x 120 with exchange and gradient polish."""
    dt = 0.002
    line = make_line(n_cmp=n_cmp, dcmp=12.5, offsets=OFF_120, ns=ns, dt=dt, n_events=n_events,
                     tau_range=(0.2, 0.93 * (ns - 1) * dt), A_range=(-4e-4, 4e-4),
                     B_range=(-1e-7, 1e-7), v_range=(1500.0, 4000.0), snr=2.0, seed=seed)
    prob = line_problem(line, half_window=5, ap_half=ap_half, cmps=cmps, t0_range=t0_range)
    de = DEConfig(np=np_, ng=ng, F=0.5, CR=0.9, seed=seed, lo=CRS_LO, hi=CRS_HI,
                  exch_every=10, polish_steps=5, polish_lr=POLISH_LR)
    return Workload(f"large_line_{n_cmp}x120x{ns}_bf16", line.traces, line.mid, line.off, dt,
                    prob, de, storage="bf16", line=line)


def random_points(line: Line, n: int, seed: int, *, ap_half: int = 0, m0_spread: float = 125.0):
    """Random (m0, it0, theta) evaluation points on a one-CMP or line gather
    for gradient checks: m0 within +-m0_spread of a CMP, theta uniform in the
    CRS bounds. Returns a Problem with one domain per point and theta [n,1,3]."""
    rng = np.random.default_rng(seed)
    c = rng.integers(0, line.n_cmp, n)
    m0 = line.cmp_x[c] + rng.uniform(-m0_spread, m0_spread, n)
    it0 = rng.integers(0, line.ns, n).astype(np.int32)
    ptr, idx = [0], []
    for ci in c:
        c0, c1 = max(0, ci - ap_half), min(line.n_cmp - 1, ci + ap_half)
        idx.append(np.arange(c0 * line.n_off, (c1 + 1) * line.n_off, dtype=np.int32))
        ptr.append(ptr[-1] + idx[-1].size)
    prob = Problem(op=CRS, half_window=5, group_m0=m0.astype(np.float32),
                   group_dt=np.full(n, line.dt, np.float32), ap_ptr=np.array(ptr, np.int32),
                   ap_idx=np.concatenate(idx), dom_it0=it0,
                   dom_group=np.arange(n, dtype=np.int32))
    lo, hi = np.array(CRS_LO), np.array(CRS_HI)
    theta = (lo + rng.uniform(0, 1, (n, 1, 3)) * (hi - lo)).astype(np.float32)
    return prob, theta
