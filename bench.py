"""Benchmark: the whole traveltime-parameter search on the 200-CMP line.

One step = one complete search (tt_search) over every zero-offset sample of
a 200-CMP x 48-offset x 1500-sample line (300,000 domains): DE with NP = 64,
NG = 100, F = 0.5, CR = 0.9, the neighbour exchange every 10 generations
and 5 gradient-polish steps, i.e. every row of the hot path. Inputs are
resident on the device when the timed region starts; between timed steps
L2 is flushed by writing a 256 MiB buffer (the line itself, 59 MB, fits in
L2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torchrun): the line is cut into N contiguous slabs of
CMPs, one per rank (tt_search_slab): each GPU holds its slab's traces plus
a read-only halo of the aperture radius, and at every exchange generation
the ranks swap the bests of their edge rows by NCCL point-to-point; the
slabs together solve the same line, so scaling is strong. (The other
workloads run as independent replicas per rank, weak scaling.) Rank 0 prints
one JSON line.

--impl reference times the CPU oracle (FP64 semblance, FP32 DE) on the host
cores instead, each step a bounded sample of the same workload.

Beside the headline line (rank 0, N = 1) the JSON carries a `comparison`:
the same search in its plain FP32 form (scalar kernel, no polish) and with
BF16-stored traces; the large line's central 100-CMP slab with BF16 and
FP32 storage and the error of its reported S against the FP64 oracle on a
1% sample of domains; and the 4096-problem batched workload with the
autotuned kernel against the scalar one. --paper-compare adds a re-run of
the paper's ENS-versus-JADE experiment (context only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ZO samples solved/s (CRS search with neighbour exchange + gradient polish)"
UNIT = "ZO samples/s"
# Algorithmic FP32 work per (trace, parameter vector) pair of K1, two counts:
#  * flops, an FMA counting 2 and the square root and its clamp 1 each:
#    traveltime 9 (CRS; CMP 5, FO-CRS 15), interpolation 33, stack 11,
#    energy 22 -> 75 for CRS;
#  * operations, an FMA counting 1 (the count 8 + 4 (2w + 1) + 1 square root
#    = 53 for CRS at w = 5: traveltime 8, per window sample an interpolation
#    product and FMA, a stack add and an energy FMA).
FLOPS_PER_TRACE_EVAL = {0: 71, 1: 75, 2: 81}  # by operator: CMP, CRS, FO-CRS
OPS_PER_TRACE_EVAL = {0: 49, 1: 53, 2: 59}
FP32_LANES = 128          # FP32 lanes per SM (an FMA per lane per clock)
L1_BYTES_PER_CLK = 128    # L1 / shared-memory data path per SM per clock


def workload_config(wl, n_gpus):
    p = wl.problem
    if wl.info is not None:
        name = (f"{p.n_groups} uneven CRS problems, 16-240 traces and 750-3000 samples "
                f"(dt 2/4 ms) each, every sample a domain, window 11")
    elif wl.storage == "bf16" and p.n_m0 and wl.line is not None and wl.line.n_cmp == 2000:
        name = (f"large line 2000 CMP x 120 offsets x 2000 samples (dt 2 ms, BF16-stored), "
                f"aperture +-25 CMP, window 11, central {p.n_m0}-CMP slab solved")
    elif p.op == 2:
        name = ("FO-CRS on the common-offset section at h0 = 1000 m of the 200-CMP x 48 x "
                "1500-sample line (dt 4 ms), aperture +-8 CMP x +-1000 m, window 11")
    else:
        sub = "" if p.n_m0 in (0, 200) else f" (first {p.n_m0} CMPs solved)"
        name = ("CRS line 200 CMP x 48 offsets x 1500 samples (dt 4 ms), aperture +-10 CMP, "
                "window 11" + sub)
    return {"workload": name,
            "n_dom": p.n_dom, "np": wl.de.np, "ng": wl.de.ng, "exch_every": wl.de.exch_every,
            "polish_steps": wl.de.polish_steps, "storage": wl.storage,
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": ("1 GPU" if n_gpus == 1 else
                            f"midpoint slabs x{n_gpus} (edge-row exchange)"
                            if getattr(wl, "slab", None) else f"replicas x{n_gpus}")}


# ------------------------------------------------------------------ ranks

def rank_env():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value any rank holds (the job finishes with its slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    """The sum of a value over the ranks (whole-job counts)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(n_dom_per_rank: int, world: int, seconds_per_step: float) -> float:
    """Whole-job ZO samples/s: every rank solves its own line of n_dom samples."""
    return world * n_dom_per_rank / seconds_per_step


# ------------------------------------------------------------------ accuracy

def recovery(wl, best_theta, tol=0.01, cmp_stride=None, sep_s=0.1, min_amp=0.7):
    """Recovered CRS parameters against the exact recentred values at
    event-centred domains: by default at each strong event's own CMP
    (|amplitude| >= min_amp); with ``cmp_stride``, at every cmp_stride-th
    solved CMP for every event (a slab of a long line crosses many events
    away from their own CMPs). A point counts when the truth (A, B, C) lies
    inside the bounds, 20 samples inside the record, and no other event's
    zero-offset time at that CMP is within sep_s seconds. Reports how many
    have A and B within ``tol`` of their bound ranges, C within ``tol``
    relative, and all three at once. B's effect on the data is tiny on
    short apertures, so its error is also given as the traveltime shift it
    causes at the aperture's farthest midpoint, |dB| dm_max^2 / (2 t0), in
    samples (median and maximum over the points), beside the shift of B's
    whole bound range."""
    import synth
    prob, line = wl.problem, wl.line
    if line is None or prob.n_m0 * prob.n_t0 != prob.n_dom:
        return None
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    ev = line.events
    hits = {"A": 0, "B": 0, "C": 0, "all": 0}
    tried, shift, b_range_shift = 0, [], []
    solved = [int(np.argmin(np.abs(line.cmp_x - m))) for m in np.unique(prob.group_m0)]
    for e in range(len(ev)):
        if cmp_stride:
            cands = solved[::cmp_stride]
        elif abs(ev[e, 5]) >= min_amp:
            cands = [int(np.argmin(np.abs(line.cmp_x - ev[e, 0])))]
        else:
            cands = []
        for c in cands:
            if c < 15 or c > line.n_cmp - 16:
                continue
            truth = synth.crs_recentre(ev[e], line.cmp_x[c])
            if truth is None or not all(lo[k] < truth[1 + k] < hi[k] for k in range(3)):
                continue
            it = int(round(truth[0] / wl.dt))
            others = [synth.crs_recentre(ev[k], line.cmp_x[c]) for k in range(len(ev)) if k != e]
            if it < 20 or it > prob.n_t0 - 20 or any(
                    o is not None and abs(o[0] - truth[0]) < sep_s for o in others):
                continue
            # the domain of (CMP c, sample it); c indexes the line, and the
            # problem may solve a slab of it
            rows = np.nonzero(np.abs(prob.group_m0 - line.cmp_x[c]) < 1e-3)[0]
            cand = np.nonzero(np.isin(prob.dom_group, rows) & (prob.dom_it0 == it))[0]
            if cand.size == 0:
                continue  # the CMP lies outside the solved slab
            d = int(cand[0])
            g = int(prob.dom_group[d])
            idx = prob.ap_idx[prob.ap_ptr[g]:prob.ap_ptr[g + 1]]
            dm_max = float(np.max(np.abs(wl.mid[idx] - prob.group_m0[g]))) if idx.size else 0.0
            tried += 1
            ok_a = abs(best_theta[d, 0] - truth[1]) <= tol * (hi[0] - lo[0])
            ok_b = abs(best_theta[d, 1] - truth[2]) <= tol * (hi[1] - lo[1])
            ok_c = abs(best_theta[d, 2] - truth[3]) <= tol * truth[3]
            hits["A"] += int(ok_a)
            hits["B"] += int(ok_b)
            hits["C"] += int(ok_c)
            hits["all"] += int(ok_a and ok_b and ok_c)
            shift.append(abs(best_theta[d, 1] - truth[2]) * dm_max ** 2 / (2 * truth[0]) / wl.dt)
            b_range_shift.append((hi[1] - lo[1]) * dm_max ** 2 / (2 * truth[0]) / wl.dt)
    out = {"within_1pct": hits, "of": tried,
           "rule": "A, B: 1% of the bound range; C: 1% relative",
           "points": (f"every {cmp_stride}th solved CMP, every event" if cmp_stride else
                      f"each event's own CMP, |amplitude| >= {min_amp}") +
                     f"; no other event within {sep_s:g} s"}
    if shift:
        out["B_edge_shift_samples"] = {"median": float(np.median(shift)),
                                       "max": float(np.max(shift)),
                                       "whole_B_range_median": float(np.median(b_range_shift))}
    return out


def fo_recovery(wl, best_theta):
    """FO-CRS: event-centred samples (CMPs within 40 m of an isolated strong
    event's midpoint) whose two slopes (Am, Ah) are within 1% and 5% of their
    bound ranges of the exact re-expansion about (m0, h0)."""
    import synth
    prob, line = wl.problem, wl.line
    lo, hi = np.array(wl.de.lo), np.array(wl.de.hi)
    h0 = float(prob.group_h0[0])
    h1 = h5 = tried = 0
    ev = line.events
    for e in range(len(ev)):
        others = np.delete(ev[:, 1], e)
        if not (np.all(np.abs(others - ev[e, 1]) > 0.1) and abs(ev[e, 5]) > 0.6):
            continue
        for c in range(3, min(line.n_cmp - 3, prob.n_m0)):
            if abs(line.cmp_x[c] - ev[e, 0]) > 40:
                continue
            p = synth.gathers.fo_recentre(ev[e], line.cmp_x[c], h0)
            if p is None:
                continue
            it = int(round(p[0] / wl.dt))
            if not 10 <= it < prob.n_t0 - 10:
                continue
            d = c * prob.n_t0 + it
            tried += 1
            err = max(abs(best_theta[d, k] - p[1 + k]) / (hi[k] - lo[k]) for k in (0, 1))
            h1 += int(err <= 0.01)
            h5 += int(err <= 0.05)
    return {"slopes_within_1pct": h1, "slopes_within_5pct": h5, "of": tried}


# ------------------------------------------------------------------ paper comparison

def paper_compare(tt, wl, dev, stream, runs=None, recover=None):
    """The paper's own experiment (Sec. 5.2-5.3, Fig. rms_coherence and
    ens_jade_execution_time) on this line: JADE (the plain search with the
    adaptation of F and CR and the archive, mu starting at 0.5, no exchange
    or polish) at 5x1, 30x30 and 80x80 against the ENS sweep at 5x1, 30x30
    and 80x80 (NP_bf 5, NG_bf 1, N_skip 2, N_cycle 1, buckets of 64 traces).
    Each search runs once untimed (graph capture) and once timed; quality is
    the RMS of the coherence panel (the paper's g-type measure) and the
    recovery of event-centred parameters."""
    import copy
    import torch
    out = {}
    runs = runs or (("jade_5x1", "jade", 5, 1), ("jade_30x30", "jade", 30, 30),
                    ("jade_80x80", "jade", 80, 80), ("ens_5x1", "ens", 5, 1),
                    ("ens_30x30", "ens", 30, 30), ("ens_80x80", "ens", 80, 80))
    recover = recover or recovery
    for label, kind, npop, ngen in runs:
        de = copy.copy(wl.de)
        de.np, de.ng, de.exch_every, de.polish_steps = max(npop, 5), ngen, 0, 0
        if kind == "jade":
            de.adapt, de.F, de.CR = 1, 0.5, 0.5
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, de, device=dev)

        def run():
            if kind == "jade":
                return tt.tt_search(ctx)
            return tt.tt_ens_search(ctx, npop, ngen, 5, 1, 2, 1, 64)

        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        th, S, n = run()
        b.record(stream)
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        S = S.cpu().numpy().astype(np.float64)
        out[label] = {"seconds": secs, "zo_samples_per_s": wl.problem.n_dom / secs,
                      "calls_per_sample": n / wl.problem.n_dom,
                      "rms_coherence": float(np.sqrt(np.mean(S * S))),
                      "recovery": recover(wl, th.cpu().numpy())}
        ctx.close()
    out["jade_30x30_over_ens_5x1_time"] = out["jade_30x30"]["seconds"] / out["ens_5x1"]["seconds"]
    if "ens_30x30" in out:
        out["jade_30x30_over_ens_30x30_time"] = (out["jade_30x30"]["seconds"] /
                                                 out["ens_30x30"]["seconds"])
    if "ens_80x80" in out:
        out["jade_80x80_over_ens_80x80_time"] = (out["jade_80x80"]["seconds"] /
                                                 out["ens_80x80"]["seconds"])
    return out


# ------------------------------------------------------------------ other workloads

def _timed_search(tt, ctx, stream, out_t=None, out_s=None):
    """One tt_search timed with CUDA events on the launching stream (the
    caller has warmed the kernels); returns (seconds, best_theta, best_S)."""
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    th, S, _ = tt.tt_search(ctx, out_t, out_s)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3, th, S


def _autotune(tt, ctx, n_dom, np_, D, dev):
    import torch
    th = torch.empty((n_dom, np_, D), dtype=torch.float32, device=dev)
    tt.tt_de_step(ctx, 0, th)
    tuned = {f"{k}/{b}": round(v, 3) for (k, b), v in tt.tt_ctx_autotune(ctx, th).items()}
    del th
    return tuned, f"{tt.tt_ctx_get_option(ctx, 'kernel')}/{tt.tt_ctx_get_option(ctx, 'block')}"


def ens_compare(tt, wl, dev, stream):
    """The ENS sweep (tt_ens_search, Sec. 3.3-3.6) on the same line at the
    paper's cheapest setting, NP_f 5 x NG_f 1, NP_bf 5 x NG_bf 1, N_skip 2,
    N_cycle 1, buckets of 64 traces: one graph-capturing run, then the median
    of five timed replays, with the call count, the RMS of the semblance
    panel and the recovery of the event-centred parameters."""
    import copy
    import torch
    de = copy.copy(wl.de)
    de.np, de.ng, de.exch_every, de.polish_steps = 5, 1, 0, 0
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, wl.problem, de, device=dev)
    tt.tt_ens_search(ctx, 5, 1, 5, 1, 2, 1, 64)
    ts = []
    for _ in range(5):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        th, S, n = tt.tt_ens_search(ctx, 5, 1, 5, 1, 2, 1, 64)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    secs = float(np.median(ts))
    S = S.cpu().numpy().astype(np.float64)
    out = {"setting": "NP 5 x NG 1 both ways, N_skip 2, N_cycle 1, buckets of 64 traces",
           "seconds": secs, "value": wl.problem.n_dom / secs,
           "calls_per_sample": n / wl.problem.n_dom,
           "rms_coherence": float(np.sqrt(np.mean(S * S))),
           "recovery": recovery(wl, th.cpu().numpy())}
    ctx.close()
    return out


def large_slab_compare(tt, dev, stream, n_slab=100, sample_frac=0.01):
    """The large line (2000 CMPs x 120 offsets x 2000 samples at 2 ms, 60
    events, SNR 2, aperture +-25 CMPs, DE 96 x 120 with exchange and polish):
    the central n_slab-CMP slab solved with BF16-stored and with FP32-stored
    traces (each autotuned, one timed search), ZO samples/s and recovery of
    each, and the error of the reported S against the FP64 oracle on a seeded
    sample of sample_frac of the slab's domains: against the FP32 record
    (what BF16 storage costs, bar 2e-3) and, for BF16, against the
    BF16-rounded record (the arithmetic alone, bar 1e-5)."""
    import oracle
    import torch
    from synth import configs
    c0 = 1000 - n_slab // 2
    wl = configs.large_line(0, cmps=list(range(c0, c0 + n_slab)))
    prob = wl.problem
    rng = np.random.default_rng(5)
    doms = np.sort(rng.choice(prob.n_dom, max(1, int(round(sample_frac * prob.n_dom))),
                              replace=False))
    out = {"workload": f"large line 2000 CMP x 120 x 2000 (dt 2 ms), central {n_slab}-CMP "
                       f"slab ({prob.n_dom} domains), aperture +-25 CMP, DE "
                       f"{wl.de.np} x {wl.de.ng}, exchange every {wl.de.exch_every}, "
                       f"{wl.de.polish_steps} polish steps",
           "s_error_sample": f"{doms.size} domains ({100 * sample_frac:g}% of the slab, seed 5)"}
    bf16_rec = None
    for storage in ("bf16", "f32"):
        ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, storage=storage,
                               device=dev)
        tuned, kern = _autotune(tt, ctx, prob.n_dom, wl.de.np, ctx.D, dev)
        secs, th, S = _timed_search(tt, ctx, stream)
        th, S = th.cpu().numpy(), S.cpu().numpy()
        ctx.close()
        ref = oracle.semblance.semblance_many(wl.traces, wl.mid, wl.off, prob,
                                              th[doms][:, None, :], domains=doms)[:, 0]
        err = np.abs(S[doms] - ref)
        e = {"value": prob.n_dom / secs, "seconds": secs, "kernel": kern,
             "recovery": recovery(wl, th, cmp_stride=5, sep_s=0.05),
             "s_error_vs_fp64_oracle": {"max": float(err.max()), "median": float(np.median(err)),
                                        "record": "FP32"}}
        if storage == "bf16":
            if bf16_rec is None:
                bf16_rec = torch.from_numpy(wl.traces).to(torch.bfloat16).to(
                    torch.float32).numpy()
            ref_b = oracle.semblance.semblance_many(bf16_rec, wl.mid, wl.off, prob,
                                                    th[doms][:, None, :], domains=doms)[:, 0]
            err_b = np.abs(S[doms] - ref_b)
            e["s_error_vs_fp64_oracle_bf16_record"] = {"max": float(err_b.max()),
                                                       "median": float(np.median(err_b))}
        out[f"{storage}_stored"] = e
    out["bf16_over_f32"] = out["bf16_stored"]["value"] / out["f32_stored"]["value"]
    return out


def batched_compare(tt, dev, stream):
    """The batched workload (4096 uneven CRS problems, 16-240 traces and
    750-3000 samples at 2 or 4 ms each, every sample a domain, DE 64 x 80):
    one timed search with the autotuned kernel against the plain form (scalar kernel, one
    pair per thread, grid-mapped), on the same context and inputs; the two
    give identical results, so they are at the same accuracy."""
    from synth import configs
    wl = configs.batched(0)
    prob = wl.problem
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, device=dev)
    tuned, kern = _autotune(tt, ctx, prob.n_dom, wl.de.np, ctx.D, dev)
    secs, th_a, _ = _timed_search(tt, ctx, stream)
    th_a = th_a.cpu().numpy()
    tt.tt_ctx_set_option(ctx, "kernel", "scalar")
    tt.tt_search(ctx)  # capture the scalar form's graph
    secs_s, th_s, _ = _timed_search(tt, ctx, stream)
    same = bool(np.array_equal(th_a, th_s.cpu().numpy()))
    ctx.close()
    return {"workload": f"{prob.n_groups} uneven CRS problems (16-240 traces, 750-3000 "
                        f"samples, dt 2/4 ms), {prob.n_dom} domains, DE {wl.de.np} x {wl.de.ng}",
            "autotuned": {"value": prob.n_dom / secs, "seconds": secs, "kernel": kern,
                          "autotune_ms": tuned},
            "plain_scalar": {"value": prob.n_dom / secs_s, "seconds": secs_s,
                             "kernel": "scalar (one pair per thread, grid-mapped)"},
            "speedup": secs_s / secs, "identical_results": same}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_median": float(np.median([float(r[3]) for r in rows
                                                   if r[3].replace(".", "").isdigit()] or [0]))}


# ------------------------------------------------------------------ oracle legs

def oracle_sample(wl, n_m0=2, n_t0=2, c0=99, it0=600):
    """A bounded sample of the workload for the CPU oracle: an n_m0 x n_t0
    block of domains in the middle of the line, with the full search
    settings (exchange inside the block)."""
    import synth
    return synth.line_problem(wl.line, half_window=5, ap_half=10,
                              cmps=list(range(c0, c0 + n_m0)), t0_range=(it0, it0 + n_t0))


def time_oracle(wl, prob):
    import oracle
    t = time.perf_counter()
    oracle.search.search(wl.traces, wl.mid, wl.off, prob, wl.de)
    return time.perf_counter() - t


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return 0
    from synth import configs
    wl = configs.crs_line(0)
    prob = oracle_sample(wl, 1, 2)
    for _ in range(args.warmup):
        time_oracle(wl, prob)
    ts = [time_oracle(wl, prob) for _ in range(args.steps)]
    per = float(np.mean(ts))
    value = prob.n_dom / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{prob.n_dom} domains (1 CMP x 2 samples at CMP 99, "
                                       "it0 600-601) per step, full NP/NG/exchange/polish"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg

# DRAM bytes (read + write) of one generation launch of K1 on the CRS line,
# packed/128, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of three launches, caches flushed by ncu before each):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:k_semblance -s 40 -c 3
#       python bench.py --steps 1 --warmup 0 --no-e2e --no-cpu-baseline --no-compare
# with the members in window order (mean of three generation launches):
# 375.0 MB read + 63.5 MB written: the compulsory bytes (theta 230.4 MB, the
# 57.6 MB line and the 76.8 MB slot map read, S 76.8 MB written, part of it
# still in L2 when the launch ends), no re-reads.
K1_LINE_DRAM_BYTES = 374_962_517 + 63_500_629
K1_LINE_DRAM_KERNEL = "packed/128"
K1_LINE_DRAM_MEMBER_ORDER = True  # the capture's launch form: members in window order


def member_order_on(tt, ctx, prob):
    """Whether the search evaluates members in window order: the option, or
    for "auto" the library's rule (mean aperture of at least 768 traces)."""
    opt = tt.tt_ctx_get_option(ctx, "member_order")
    if opt == "auto":
        ap = np.diff(np.asarray(prob.ap_ptr))[np.asarray(prob.dom_group)]
        return bool(ap.size) and float(ap.mean()) >= 768.0
    return bool(opt)


def hbm_peak_gbs():
    """The measured HBM copy bandwidth of this GPU model (MEASURED_PEAKS.json
    at the repository root), else the fallback figure of an earlier GB300
    measurement."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def l2_probe(dev, stream):
    """L2 bandwidth probe: device-to-device copies between two buffers that
    together fit in L2, 20 copies captured in a CUDA graph (no launch gaps
    from the host), replayed after warm-up and timed with CUDA events; the
    largest read + write rate over three sizes. The semblance kernel's own L2
    traffic is small (L1 serves ~99% of its loads), so this bounds nothing on
    the line: it places the L2 level next to the L1 and HBM figures."""
    import torch
    best = 0.0
    for mib in (16, 24, 32):
        n = mib << 18
        a = torch.ones(n, dtype=torch.float32, device=dev)
        b = torch.empty_like(a)
        b.copy_(a)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(20):
                b.copy_(a)
        with torch.cuda.stream(stream):
            g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                g.replay()
            e1.record(stream)
        e1.synchronize()
        best = max(best, 2 * n * 4 * 100 / (e0.elapsed_time(e1) / 1e3) / 1e9)
        del g, a, b
    return {"gbs": best, "method": "torch copy_ between two L2-resident buffers (2 x 16-32 MiB), "
                                   "20 copies per CUDA graph, 5 replays, read + write bytes"}


def device_counts(ctx_sm):
    """(SM count, maximum SM clock in MHz and where it came from): the SM
    count is the library's query of the device; the clock is nvidia-smi's
    clocks.max.sm, else the measured-peaks file's sm_max_mhz."""
    mhz, src = None, None
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,"
                              "nounits", "-i", os.environ.get("LOCAL_RANK", "0")],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        mhz, src = float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except (OSError, KeyError, ValueError):
            mhz, src = None, "unknown"
    return int(ctx_sm), mhz, src


def roofline(tt, ctx, prob, stats, args, clk, stream):
    """Roofline of K1 from the library's live CUDA-event timing of every
    semblance launch in the timed steps. The bound is the on-chip data path
    that K1's window loads go through: every (trace, vector) pair gathers
    2w + 2 samples (48 B in FP32, 24 B in BF16) with 4-byte loads that hit
    in L1, so
      achieved = pairs per launch x bytes per pair / mean launch time,
      peak = the L1 load rate the library's probe measures on this GPU with
             the same load instruction (coalesced, one cache line per warp
             request, every resident warp loading);
    beside it the derived line rate, n_sm x 128 B x max SM clock, printed
    with the SM count and clock it uses, the FP32 pipe (n_sm x 128 lanes x 2
    flops x clock) under the two work counts, and the DRAM bytes of one
    launch from an ncu capture (traffic)."""
    n_sm, mhz, mhz_src = device_counts(tt.tt_ctx_get_option(ctx, "sm_count"))
    if mhz is None:
        mhz = clk.get("sm_max_mhz") or 0.0
    w = int(prob.half_window)
    bytes_pair = (2 * w + 2) * (2 if args.storage == "bf16" else 4)
    ms_launch = stats["semblance_ms"] / stats["timed_launches"]
    pairs_launch = stats["trace_evals"] / stats["semblance_launches"]
    pairs_s = pairs_launch / (ms_launch / 1e3)
    achieved = pairs_s * bytes_pair / 1e9
    derived = n_sm * L1_BYTES_PER_CLK * mhz * 1e6 / 1e9
    probe = l1_probe(tt, ctx, stream, n_sm, mhz)
    peak = probe["gbs"]
    kern = f"{tt.tt_ctx_get_option(ctx, 'kernel')}/{tt.tt_ctx_get_option(ctx, 'block')}"
    same_form = (kern == K1_LINE_DRAM_KERNEL and
                 member_order_on(tt, ctx, prob) == K1_LINE_DRAM_MEMBER_ORDER)
    traffic = (K1_LINE_DRAM_BYTES if (args.workload == "line" and args.storage == "f32" and
                                      not args.cmps and same_form) else None)
    fp32_peak = n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12
    op = int(prob.op)
    roof = {"bound": "l1", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "kernel": f"k_semblance ({kern})",
            "peak_source": "measured: " + probe["method"],
            "l1_probe": probe,
            "derived": {"peak": derived, "frac": achieved / derived if derived else None,
                        "source": (f"{n_sm} SMs (device query) x {L1_BYTES_PER_CLK} B/clk x "
                                   f"{mhz:.0f} MHz ({mhz_src})")},
            "sm_count": n_sm, "sm_max_mhz": mhz, "bytes_per_pair": bytes_pair,
            "pairs_per_launch": pairs_launch, "per_launch_ms": ms_launch,
            "trace_evals_per_s": pairs_s, "trace_samples_per_s": pairs_s * (2 * w + 1),
            "semblance_share_of_step": None,
            "fp32": {"peak_tflops": fp32_peak,
                     "flops_fma2": {"per_pair": FLOPS_PER_TRACE_EVAL[op],
                                    "tflops": pairs_s * FLOPS_PER_TRACE_EVAL[op] / 1e12,
                                    "frac": pairs_s * FLOPS_PER_TRACE_EVAL[op] / 1e12 / fp32_peak},
                     "ops_fma1": {"per_pair": OPS_PER_TRACE_EVAL[op],
                                  "tops": pairs_s * OPS_PER_TRACE_EVAL[op] / 1e12,
                                  "peak_tops": fp32_peak / 2,
                                  "frac": pairs_s * OPS_PER_TRACE_EVAL[op] / 1e12 /
                                  (fp32_peak / 2)}}}
    # the gathered samples as a byte rate beside the HBM copy bandwidth: L1
    # serves them, at several times what HBM could deliver
    hbm, src = hbm_peak_gbs()
    roof["gathered"] = {"gbs": achieved, "hbm_gbs": hbm, "hbm_source": src,
                        "over_hbm": achieved / hbm}
    return roof


def l1_probe(tt, ctx, stream, n_sm, mhz):
    """The L1 load bandwidth measured by the library's probe (coalesced
    4-byte loads from an L1-resident window, one wave of resident blocks),
    one warm-up launch then five timed with CUDA events, also as bytes per
    clock per SM at the maximum SM clock."""
    import torch
    tt.tt_ctx_probe_l1(ctx, 200, stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    n = sum(tt.tt_ctx_probe_l1(ctx, 4000, stream) for _ in range(5))
    b.record(stream)
    torch.cuda.synchronize()
    gbs = n / (a.elapsed_time(b) / 1e3) / 1e9
    clk = n_sm * mhz * 1e6
    return {"gbs": gbs, "bytes_per_clk_per_sm": gbs * 1e9 / clk if clk else None,
            "method": "tt_ctx_probe_l1: one wave of resident 256-thread blocks, 32 coalesced 4-byte "
                      "ld.global.nc per thread per iteration from a 24 KiB window (other lines "
                      "every iteration), 5 x 4000 iterations, CUDA events; bytes per clock at "
                      "the maximum SM clock"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip every comparison entry (other forms, workloads and the ENS sweep)")
    ap.add_argument("--paper-compare", action="store_true",
                    help="also re-run the paper's ENS-vs-JADE experiment on the line (context, "
                         "off by default)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large-line slab comparison (BF16 vs FP32 storage, S error "
                         "against the FP64 oracle on a 1%% sample)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-workload comparison (autotuned vs scalar kernel)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--cmps", type=int, default=0,
                    help="solve only the first CMPS midpoints of the line (profiling case)")
    ap.add_argument("--workload", default="line", choices=["line", "batched", "fo", "large"],
                    help="line: the 200-CMP CRS line (default); batched: 4096 uneven CRS "
                         "problems (every sample a domain, DE 64 x 80, autotuned kernel); fo: "
                         "FO-CRS on the line's common-offset section at 1000 m; large: the "
                         "2000-CMP x 120 x 2000 BF16-stored line, a central slab of --cmps "
                         "CMPs (default 100) solved")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world, rank, local = rank_env()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)  # before the process group: NCCL binds this rank's GPU
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2304_11399_gb300 import build as _build
    _build.build()
    import paper_2304_11399_gb300 as tt
    from synth import configs

    if args.workload == "large":
        n_slab = args.cmps or 100
        c0 = 1000 - n_slab // 2
        wl = configs.large_line(rank, cmps=list(range(c0, c0 + n_slab)))
        args.storage = "bf16"
    else:
        wl = {"line": configs.crs_line, "batched": configs.batched,
              "fo": configs.fo_panel}[args.workload](rank)
    wl.storage = args.storage
    if args.cmps and args.workload == "line":
        import synth
        wl.problem = synth.line_problem(wl.line, half_window=5, ap_half=10,
                                        cmps=list(range(args.cmps)))
    slab = None
    if world > 1 and args.workload == "line":
        # one slab of the same line per rank, with its aperture halo
        import synth
        from paper_2304_11399_gb300.slab import halo_exchange
        wl = configs.crs_line(0)
        c0, c1 = synth.slab_bounds(wl.problem.n_m0, world, rank,
                                   weights=np.diff(wl.problem.ap_ptr))  # equal work
        wl.traces, wl.mid, wl.off, wl.problem, base, hp, hn = synth.slab_problem(
            wl.line, c0, c1, half_window=5, ap_half=10)
        slab = (base, hp, hn, halo_exchange(rank, world))
        wl.slab = (c0, c1)
    prob = wl.problem

    def search(ctx, best_t, best_s):
        if slab is None:
            return tt.tt_search(ctx, best_t, best_s)
        return tt.tt_search_slab(ctx, *slab, best_theta=best_t, best_S=best_s)
    # CPU baseline first (rank 0, N = 1): the oracle as it stands on a sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "line":
        sp = oracle_sample(wl)
        secs = time_oracle(wl, sp)
        cpu = {"value": sp.n_dom / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sp.n_dom} domains (2 CMP x 2 samples at CMP 99-100, it0 600-601), "
                         f"full NP/NG/exchange/polish, {secs:.1f} s single-threaded numpy"}

    stream = torch.cuda.current_stream()
    ctx = tt.tt_ctx_create(wl.traces, wl.mid, wl.off, prob, wl.de, storage=args.storage,
                           device=dev)
    # pick the kernel variant and block size on a generation-0 population
    # (every variant gives the same bits, so this changes speed only)
    th = torch.empty((prob.n_dom, wl.de.np, ctx.D), dtype=torch.float32, device=dev)
    tt.tt_de_step(ctx, 0, th)
    tuned = {f"{k}/{b}": round(v, 3) for (k, b), v in tt.tt_ctx_autotune(ctx, th).items()}
    del th
    best_t = torch.empty((prob.n_dom, ctx.D), dtype=torch.float32, device=dev)
    best_s = torch.empty((prob.n_dom,), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 18, dtype=torch.float32, device=dev)  # 256 MiB

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        search(ctx, best_t, best_s)
    barrier()
    tt.tt_ctx_profile(ctx, True)
    tt.tt_ctx_stats(ctx, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    n_evals = 0
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        _, _, n_evals = search(ctx, best_t, best_s)
        ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    stats = tt.tt_ctx_stats(ctx, reset=True)
    tt.tt_ctx_profile(ctx, False)
    ms_max = max_over_ranks(ms, world, dev)
    per_step_s = ms_max / 1e3 / args.steps
    # whole-job ZO samples: every rank's own line (replicas) or the slabs
    # of one line
    n_total = prob.n_dom * world if slab is None else int(sum_over_ranks(prob.n_dom, world,
                                                                         dev))
    value = n_total / per_step_s

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host_tr = torch.from_numpy(wl.traces).pin_memory()
        host_bt = torch.empty((prob.n_dom, ctx.D), dtype=torch.float32).pin_memory()
        host_bs = torch.empty((prob.n_dom,), dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tt.tt_ctx_load_traces(ctx, host_tr)
            search(ctx, best_t, best_s)
            host_bt.copy_(best_t, non_blocking=True)
            host_bs.copy_(best_s, non_blocking=True)
            torch.cuda.synchronize()
        barrier()
        e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": n_total / (e_s / args.steps), "unit": UNIT,
               "h2d_bytes_per_step": int(sum_over_ranks(wl.traces.nbytes, world, dev)),
               "d2h_bytes_per_step": int(sum_over_ranks(host_bt.numel() * 4 +
                                                        host_bs.numel() * 4, world, dev))}

    # roofline of the dominant kernel (semblance), from its live launch times
    roof = None
    if stats["timed_launches"] > 0 and stats["semblance_ms"] > 0:
        roof = roofline(tt, ctx, prob, stats, args, clk, stream)
        roof["semblance_share_of_step"] = stats["semblance_ms"] / ms
        if rank == 0:
            roof["l2_probe"] = l2_probe(dev, stream)
    # the same search in other forms on the same GPU (rank 0, line workload)
    comparison = None
    if rank == 0 and world == 1 and args.workload == "line" and not args.no_compare:
        import copy
        torch.cuda.synchronize()
        comparison = {"optimised_fp32": {"value": value,
                                         "recovery": recovery(wl, best_t.cpu().numpy())}}

        def one_form(label, storage, kernel, polish, note):
            w2 = copy.copy(wl)
            w2.de = copy.copy(wl.de)
            w2.de.polish_steps = polish
            c2 = tt.tt_ctx_create(w2.traces, w2.mid, w2.off, prob, w2.de, storage=storage,
                                  device=dev)
            tt.tt_ctx_set_option(c2, "kernel", kernel)
            tt.tt_ctx_set_option(c2, "search_graph", False)
            # rank 0 alone runs these: a device synchronize, not a barrier
            # across ranks
            tt.tt_search(c2, best_t, best_s)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tt.tt_search(c2, best_t, best_s)
            b.record(stream)
            torch.cuda.synchronize()
            secs = a.elapsed_time(b) / 1e3
            comparison[label] = {"value": prob.n_dom / secs, "note": note,
                                 "recovery": recovery(w2, best_t.cpu().numpy())}
            c2.close()

        one_form("plain_fp32", "f32", "scalar", 0,
                 "one (domain, individual) pair per thread, scalar FP32, no polish, eager")
        one_form("bf16_stored", "bf16", "packed", wl.de.polish_steps,
                 "BF16 trace copy, FP32 arithmetic, FP64 chunked energy, polish")
        comparison["speedup_vs_plain_fp32"] = value / comparison["plain_fp32"]["value"]
        comparison["ens_sweep"] = ens_compare(tt, wl, dev, stream)
        if not args.no_large:
            comparison["large_line_slab"] = large_slab_compare(tt, dev, stream)
        if not args.no_batched:
            comparison["batched"] = batched_compare(tt, dev, stream)
        if args.paper_compare:
            comparison["paper_ens_vs_jade"] = paper_compare(tt, wl, dev, stream)
            # the paper's experiments use FO-CRS on a common-offset 1000 m panel
            import synth
            wfo = copy.copy(wl)
            wfo.problem = synth.gathers.fo_problem(wl.line, half_window=5, h0=1000.0, ap_half=8,
                                                   off_half=1000.0)
            wfo.de = copy.copy(wl.de)
            wfo.de.lo, wfo.de.hi = configs.FO_LO, configs.FO_HI
            comparison["paper_ens_vs_jade_focrs"] = paper_compare(
                tt, wfo, dev, stream, recover=fo_recovery,
                runs=(("jade_5x1", "jade", 5, 1), ("jade_30x30", "jade", 30, 30),
                      ("ens_5x1", "ens", 5, 1)))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_s * 1e3,
                "higher_is_better": True, "scaling": "strong" if slab else "weak",
                "vs_baseline": None,
                "dtype": "f32" if args.storage == "f32" else "bf16-stored/f32",
                "data": "synthetic (seeded Ricker events + Gaussian noise, SNR 3)",
                "config": workload_config(wl, world), "clocks": clk, "e2e": e2e,
                "gpu_launches": int(stats["launches"]), "semblance_calls_per_step": n_evals,
                "roofline": roof, "cpu_baseline": cpu, "comparison": comparison}
        line["config"]["member_order"] = member_order_on(tt, ctx, prob)
        if tuned:
            line["config"]["autotune_ms"] = tuned
            line["config"]["kernel"] = (f"{tt.tt_ctx_get_option(ctx, 'kernel')}/"
                                        f"{tt.tt_ctx_get_option(ctx, 'block')}")
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
