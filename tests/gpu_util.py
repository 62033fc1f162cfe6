"""Shared helpers of the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np
import torch

import synth
from synth import configs


def dev():
    return torch.device("cuda:0")


def random_theta(n_dom, P, lo, hi, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    return (lo + rng.uniform(0, 1, (n_dom, P, lo.size)) * (hi - lo)).astype(np.float32)


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev())


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest even) and back, via torch."""
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(
        torch.float32).numpy()


def small_line(seed=0, **kw):
    kw.setdefault("n_cmp", 12)
    kw.setdefault("ns", 200)
    kw.setdefault("n_events", 6)
    kw.setdefault("ap_half", 3)
    kw.setdefault("tau_max", 0.7)
    return configs.crs_line(seed, **kw)


__all__ = ["dev", "random_theta", "to_dev", "bf16_round", "small_line", "synth", "configs"]
