"""Synthetic prestack gathers, geometry and domain lists (numpy, seeded).

Data model
----------
A 2-D line has ``n_cmp`` common-midpoint (CMP) positions ``m = x0 + c*dcmp``
and, at each, ``n_off`` traces with full source-receiver offsets ``h``.
Traces are stored trace-major and sorted by (CMP, offset), the
offset-midpoint ordering the paper uses to keep similar domains adjacent
(Sec. "Evolution by neighborhood similarity").

Each reflection event ``e`` is a traveltime surface about a midpoint m_e,

    t_e(m, h)^2 = (tau_e + A_e (m - m_e))^2 + B_e (m - m_e)^2 + C_e h^2 ,

carrying a zero-phase Ricker wavelet of peak frequency ``freq`` (no
stretch) and amplitude ``amp_e``. Gaussian noise is added with standard
deviation (peak |noise-free amplitude|) / SNR. Where the right-hand side is
negative the event is absent from that trace.

A *domain* is one zero-offset sample (m0, it0) (the paper's (t, tr) pair,
Sec. "Traveltime parameter search"); a *group* is a set of domains sharing
one midpoint m0, sample interval and trace aperture.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CMP = 0  # operator id: CMP hyperbola, theta = (C,)
CRS = 1  # operator id: zero-offset CRS surface, theta = (A, B, C)
FOCRS = 2  # operator id: finite-offset CRS, theta = (Am, Ah, Bmm, Bmh, Bhh)


@dataclasses.dataclass
class Line:
    traces: np.ndarray      # float32 [n_tr, ns]
    mid: np.ndarray         # float32 [n_tr]  midpoint of each trace (m)
    off: np.ndarray         # float32 [n_tr]  full offset of each trace (m)
    dt: float               # s
    ns: int
    n_cmp: int
    n_off: int
    cmp_x: np.ndarray       # float64 [n_cmp] CMP positions (m)
    events: np.ndarray      # float64 [n_ev, 6]: m_e, tau, A, B, C, amp

    @property
    def n_tr(self) -> int:
        return self.traces.shape[0]


@dataclasses.dataclass
class Problem:
    """Domains, groups and apertures (CSR over trace indices)."""
    op: int
    half_window: int
    group_m0: np.ndarray    # float32 [G]
    group_dt: np.ndarray    # float32 [G]
    ap_ptr: np.ndarray      # int32 [G+1]
    ap_idx: np.ndarray      # int32 [nnz] trace indices
    dom_it0: np.ndarray     # int32 [n_dom]
    dom_group: np.ndarray   # int32 [n_dom]
    n_m0: int = 0           # exchange grid: domains laid out m0-major,
    n_t0: int = 0           # d = im0 * n_t0 + it0 (0 if no grid)
    group_h0: np.ndarray | None = None  # float32 [G] central offset (FO-CRS only)

    @property
    def n_dom(self) -> int:
        return int(self.dom_it0.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.group_m0.shape[0])

    @property
    def dim(self) -> int:
        return {CMP: 1, CRS: 3, FOCRS: 5}[self.op]

    def aperture(self, g: int) -> np.ndarray:
        return self.ap_idx[self.ap_ptr[g]:self.ap_ptr[g + 1]]


def ricker(tau: np.ndarray, freq: float) -> np.ndarray:
    a = (math.pi * freq * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _add_events(traces, mid, off, dt, events, freq):
    ns = traces.shape[1]
    half = int(math.ceil(0.08 / dt))
    rows = np.arange(traces.shape[0])
    for m_e, tau, A, B, C, amp in events:
        dm = mid.astype(np.float64) - m_e
        h = off.astype(np.float64)
        T = (tau + A * dm) ** 2 + B * dm * dm + C * h * h
        ok = T >= 0.0
        t = np.sqrt(np.where(ok, T, 0.0))
        n0 = np.floor(t / dt).astype(np.int64)
        for l in range(-half, half + 1):
            n = n0 + l
            valid = ok & (n >= 0) & (n < ns)
            r = rows[valid]
            traces[r, n[valid]] += (amp * ricker(n[valid] * dt - t[valid], freq)).astype(np.float32)


def make_line(*, n_cmp: int, dcmp: float, offsets: np.ndarray, ns: int, dt: float,
              n_events: int, tau_range, A_range, B_range, v_range, snr: float,
              seed: int, freq: float = 25.0, x0: float = 0.0) -> Line:
    """Build a seeded synthetic 2-D line (see module docstring)."""
    rng = np.random.default_rng(seed)
    offsets = np.asarray(offsets, dtype=np.float64)
    n_off = offsets.shape[0]
    cmp_x = x0 + dcmp * np.arange(n_cmp, dtype=np.float64)
    mid = np.repeat(cmp_x, n_off).astype(np.float32)
    off = np.tile(offsets, n_cmp).astype(np.float32)
    ev = np.empty((n_events, 6))
    ev[:, 0] = rng.uniform(cmp_x[0], cmp_x[-1], n_events) if n_cmp > 1 else cmp_x[0]
    ev[:, 1] = rng.uniform(*tau_range, n_events)
    ev[:, 2] = rng.uniform(*A_range, n_events) if A_range is not None else 0.0
    ev[:, 3] = rng.uniform(*B_range, n_events) if B_range is not None else 0.0
    v = rng.uniform(*v_range, n_events)
    ev[:, 4] = 1.0 / (v * v)
    ev[:, 5] = rng.uniform(0.5, 1.0, n_events) * rng.choice([-1.0, 1.0], n_events)
    traces = np.zeros((n_cmp * n_off, ns), dtype=np.float32)
    _add_events(traces, mid, off, dt, ev, freq)
    peak = float(np.max(np.abs(traces))) if traces.size else 0.0
    if snr and peak > 0.0:
        sigma = peak / snr
        traces += (sigma * rng.standard_normal(traces.shape, dtype=np.float32)).astype(np.float32)
    return Line(traces=traces, mid=mid, off=off, dt=float(dt), ns=int(ns), n_cmp=n_cmp,
                n_off=n_off, cmp_x=cmp_x, events=ev)


def cmp_problem(line: Line, *, half_window: int, cmp_index: int = 0,
                it0=None) -> Problem:
    """CMP-operator problem on one CMP gather: one group, all its traces."""
    lo = cmp_index * line.n_off
    idx = np.arange(lo, lo + line.n_off, dtype=np.int32)
    it0 = np.arange(line.ns, dtype=np.int32) if it0 is None else np.asarray(it0, np.int32)
    return Problem(op=CMP, half_window=half_window,
                   group_m0=np.array([line.cmp_x[cmp_index]], np.float32),
                   group_dt=np.array([line.dt], np.float32),
                   ap_ptr=np.array([0, idx.size], np.int32), ap_idx=idx,
                   dom_it0=it0, dom_group=np.zeros(it0.size, np.int32),
                   n_m0=1, n_t0=int(it0.size))


def fo_problem(line: Line, *, half_window: int, h0: float, ap_half: int, off_half: float,
               cmps=None, t0_range=None) -> Problem:
    """FO-CRS problem on the common-offset section at full offset h0: one
    group per CMP, aperture = traces of the CMPs within +-ap_half with
    |h - h0| <= off_half; domains (m0, it0) laid out m0-major, it0 indexing
    the section's time t(m0, h0)."""
    cmps = np.arange(line.n_cmp) if cmps is None else np.asarray(cmps)
    t0s = np.arange(line.ns) if t0_range is None else np.arange(*t0_range)
    offs = line.off[:line.n_off].astype(np.float64)
    sel = np.nonzero(np.abs(offs - h0) <= off_half + 1e-9)[0]
    ptr = [0]
    idx = []
    for c in cmps:
        c0, c1 = max(0, c - ap_half), min(line.n_cmp - 1, c + ap_half)
        rows = (np.arange(c0, c1 + 1)[:, None] * line.n_off + sel[None, :]).ravel()
        idx.append(rows.astype(np.int32))
        ptr.append(ptr[-1] + rows.size)
    G = len(cmps)
    return Problem(op=FOCRS, half_window=half_window,
                   group_m0=line.cmp_x[cmps].astype(np.float32),
                   group_dt=np.full(G, line.dt, np.float32),
                   ap_ptr=np.array(ptr, np.int32), ap_idx=np.concatenate(idx),
                   dom_it0=np.tile(t0s.astype(np.int32), G),
                   dom_group=np.repeat(np.arange(G, dtype=np.int32), t0s.size),
                   n_m0=G, n_t0=int(t0s.size), group_h0=np.full(G, h0, np.float32))


def line_problem(line: Line, *, half_window: int, ap_half: int, cmps=None,
                 t0_range=None) -> Problem:
    """CRS problem over a line: one group per CMP, aperture = traces of the
    CMPs within +-ap_half of it (clipped at the line ends); domains laid
    out m0-major over ``cmps`` x ``t0_range``."""
    cmps = np.arange(line.n_cmp) if cmps is None else np.asarray(cmps)
    t0s = np.arange(line.ns) if t0_range is None else np.arange(*t0_range)
    ptr = [0]
    idx = []
    for c in cmps:
        c0, c1 = max(0, c - ap_half), min(line.n_cmp - 1, c + ap_half)
        idx.append(np.arange(c0 * line.n_off, (c1 + 1) * line.n_off, dtype=np.int32))
        ptr.append(ptr[-1] + idx[-1].size)
    G = len(cmps)
    return Problem(op=CRS, half_window=half_window,
                   group_m0=line.cmp_x[cmps].astype(np.float32),
                   group_dt=np.full(G, line.dt, np.float32),
                   ap_ptr=np.array(ptr, np.int32), ap_idx=np.concatenate(idx),
                   dom_it0=np.tile(t0s.astype(np.int32), G),
                   dom_group=np.repeat(np.arange(G, dtype=np.int32), t0s.size),
                   n_m0=G, n_t0=int(t0s.size))


def slab_bounds(n_m0: int, world: int, rank: int, weights=None):
    """CMPs [c0, c1) of slab ``rank`` when n_m0 CMPs are cut into ``world``
    contiguous slabs. Without ``weights`` the slabs' sizes differ by at most
    one (the first n_m0 % world slabs take the extra CMP). With ``weights``
    (the work of each CMP, e.g. its aperture's trace count: CMPs near the
    line ends have clipped apertures) the r-th cut falls where the running
    work is nearest to r / world of the total, every slab keeping at least
    one CMP, so that the slabs carry about equal work."""
    if weights is None:
        base, extra = divmod(n_m0, world)
        c0 = rank * base + min(rank, extra)
        return c0, c0 + base + (1 if rank < extra else 0)
    w = np.asarray(weights, dtype=np.float64)
    if w.shape != (n_m0,) or world > n_m0 or np.any(w < 0):
        raise ValueError("weights must give one non-negative value per CMP, world <= n_m0")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    cuts = [0]
    for r in range(1, world):
        k = int(np.argmin(np.abs(cum - r * cum[-1] / world)))
        cuts.append(min(max(k, cuts[-1] + 1), n_m0 - (world - r)))
    cuts.append(n_m0)
    return cuts[rank], cuts[rank + 1]


def slab_problem(line: Line, c0: int, c1: int, *, half_window: int, ap_half: int):
    """The inputs of one slab of a sharded line search: the CRS problem of
    CMPs [c0, c1) (every sample a domain, m0-major) over a copy of only the
    traces its apertures read -- the slab's own CMPs plus a read-only halo
    of ap_half CMPs on each side, clipped at the line ends -- with the
    aperture lists re-indexed into that copy (same traces, same order).
    Returns (traces, mid, off, problem, dom_base, has_prev, has_next):
    dom_base is the global index of the slab's first domain on the whole
    line's m0-major grid; has_prev / has_next say whether CMPs exist before
    c0 / from c1 on."""
    prob = line_problem(line, half_window=half_window, ap_half=ap_half,
                        cmps=list(range(c0, c1)))
    h0 = max(0, c0 - ap_half) * line.n_off
    h1 = min(line.n_cmp, c1 + ap_half) * line.n_off
    prob.ap_idx = (prob.ap_idx - h0).astype(np.int32)
    return (np.ascontiguousarray(line.traces[h0:h1]), line.mid[h0:h1].copy(),
            line.off[h0:h1].copy(), prob, c0 * line.ns, c0 > 0, c1 < line.n_cmp)


def batched_problems(*, n_prob: int, ntr_range, ns_range, dts, seed: int,
                     n_events: int = 8, snr: float = 5.0, ap_cmp: int = 10,
                     dcmp: float = 12.5, doff: float = 50.0, max_off: float = 2350.0,
                     tau_range=(0.2, 1.9), A_range=(-4e-4, 4e-4), B_range=(-1e-7, 1e-7),
                     v_range=(1500.0, 4000.0), domains_per_problem=None):
    """Many independent CRS problems with uneven trace and sample counts.

    Problem p has N_p ~ U[ntr_range] traces at random midpoints on a
    ``dcmp`` grid within +-``ap_cmp`` CMPs of its centre and random offsets
    on a ``doff`` grid in [0, max_off]; NT_p ~ U[ns_range] samples at
    dt_p drawn from ``dts``. All traces are packed into one trace-major
    array of width max NT_p, zero beyond each problem's NT_p (the record is
    zero outside its samples, so the padding changes no value). Every
    sample of a problem is a domain unless ``domains_per_problem`` caps it.
    Returns (traces, mid, off, problem, per-problem info dict).
    """
    rng = np.random.default_rng(seed)
    ntr = rng.integers(ntr_range[0], ntr_range[1] + 1, n_prob)
    nsp = rng.integers(ns_range[0], ns_range[1] + 1, n_prob)
    dtp = rng.choice(np.asarray(dts, np.float64), n_prob)
    ns_max = int(nsp.max())
    n_tr = int(ntr.sum())
    traces = np.zeros((n_tr, ns_max), np.float32)
    mid = np.empty(n_tr, np.float32)
    off = np.empty(n_tr, np.float32)
    ptr = np.zeros(n_prob + 1, np.int64)
    ptr[1:] = np.cumsum(ntr)
    m0 = np.empty(n_prob, np.float64)
    events = []
    it0s, groups = [], []
    for p in range(n_prob):
        lo, hi = int(ptr[p]), int(ptr[p + 1])
        m0[p] = 0.0  # problems are independent; a common origin keeps FP32 coordinates exact
        mid[lo:hi] = m0[p] + dcmp * rng.integers(-ap_cmp, ap_cmp + 1, hi - lo)
        off[lo:hi] = doff * rng.integers(0, int(max_off // doff) + 1, hi - lo)
        ns_p, dt_p = int(nsp[p]), float(dtp[p])
        ev = np.empty((n_events, 6))
        ev[:, 0] = m0[p]
        ev[:, 1] = rng.uniform(*tau_range, n_events)
        ev[:, 2] = rng.uniform(*A_range, n_events)
        ev[:, 3] = rng.uniform(*B_range, n_events)
        v = rng.uniform(*v_range, n_events)
        ev[:, 4] = 1.0 / (v * v)
        ev[:, 5] = rng.uniform(0.5, 1.0, n_events) * rng.choice([-1.0, 1.0], n_events)
        block = np.zeros((hi - lo, ns_p), np.float32)
        _add_events(block, mid[lo:hi], off[lo:hi], dt_p, ev, 25.0)
        peak = float(np.max(np.abs(block)))
        if snr and peak > 0:
            block += (peak / snr * rng.standard_normal(block.shape, dtype=np.float32))
        traces[lo:hi, :ns_p] = block
        events.append(ev)
        nd = ns_p if domains_per_problem is None else min(ns_p, domains_per_problem)
        sel = np.arange(ns_p) if nd == ns_p else np.sort(rng.choice(ns_p, nd, replace=False))
        it0s.append(sel.astype(np.int32))
        groups.append(np.full(nd, p, np.int32))
    prob = Problem(op=CRS, half_window=5, group_m0=m0.astype(np.float32),
                   group_dt=dtp.astype(np.float32), ap_ptr=ptr.astype(np.int32),
                   ap_idx=np.arange(n_tr, dtype=np.int32),
                   dom_it0=np.concatenate(it0s), dom_group=np.concatenate(groups))
    info = dict(ntr=ntr, ns=nsp, dt=dtp, events=events, ns_max=ns_max)
    return traces, mid, off, prob, info


def fo_recentre(event, m0: float, h0: float):
    """Exact FO-CRS parameters of an event surface re-expanded about the
    central point (m0, h0) of a common-offset section.

    With Dc = m0 - m_e, t^2 = (tau + A Dc + A dm)^2 + B (Dc + dm)^2 +
    C (h0 + dh)^2 is the quadratic c00 + c10 dm + c01 dh + c20 dm^2 +
    c02 dh^2 (no dm dh term) with c00 = (tau + A Dc)^2 + B Dc^2 + C h0^2,
    c10 = 2 A (tau + A Dc) + 2 B Dc, c01 = 2 C h0, c20 = A^2 + B, c02 = C.
    Matching (t0 + Am dm + Ah dh)^2 + Bmm dm^2 + Bmh dm dh + Bhh dh^2 term by
    term: t0 = sqrt(c00), Am = c10 / (2 t0), Ah = c01 / (2 t0),
    Bmm = c20 - Am^2, Bmh = -2 Am Ah, Bhh = c02 - Ah^2. Returns
    (t0, Am, Ah, Bmm, Bmh, Bhh) or None where c00 <= 0."""
    m_e, tau, A, B, C = (float(v) for v in event[:5])
    dc = m0 - m_e
    c00 = (tau + A * dc) ** 2 + B * dc * dc + C * h0 * h0
    if c00 <= 0.0:
        return None
    t0 = math.sqrt(c00)
    Am = (A * (tau + A * dc) + B * dc) / t0
    Ah = C * h0 / t0
    return t0, Am, Ah, A * A + B - Am * Am, -2.0 * Am * Ah, C - Ah * Ah


def crs_recentre(event, m0: float):
    """Exact ZO-CRS parameters of an event surface re-expanded about m0.

    The event's zero-offset time squared is the quadratic
    q(D) = (tau + A D)^2 + B D^2 in D = m - m_e. Writing D = Dc + d with
    Dc = m0 - m_e and collecting powers of d gives
    q = t0^2 + 2 t0 A' d + (A'^2 + B') d^2 with
    t0 = sqrt(q(Dc)), A' = ((tau + A Dc) A + B Dc) / t0, B' = A^2 + B - A'^2,
    and the offset term C h^2 is unchanged. Returns (t0, A', B', C) or None
    where q(Dc) <= 0 (no zero-offset arrival at m0).
    """
    m_e, tau, A, B, C = (float(v) for v in event[:5])
    dc = m0 - m_e
    q = (tau + A * dc) ** 2 + B * dc * dc
    if q <= 0.0:
        return None
    t0 = math.sqrt(q)
    Ap = ((tau + A * dc) * A + B * dc) / t0
    Bp = A * A + B - Ap * Ap
    return t0, Ap, Bp, C
