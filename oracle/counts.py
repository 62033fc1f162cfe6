"""Semblance-call counts (TEST INFRASTRUCTURE).

JADE (Sec. 2.1.6, eq. jade_semblance): every one of the P_d samples starts
with NP individuals and evolves them for NG generations, so
    calls = P_d * NP * (1 + NG).

ENS (Sec. 3.6.1, eq. ens_semblance): per estimated sample the forward stage
costs S_f = NP_f (1 + NG_f); each backward-and-forward cycle initialises
only NP_bf - 1 new members, costing S_bf = 2 (NP_bf (1 + NG_bf) - 1); each
of the N_skip skipped samples costs one interpolated call per stage, of
which there are 2 N_cycle + 1; and ceil(P_d / (N_skip + 1)) samples are
estimated:
    calls = ceil(P_d / (N_skip + 1)) * (S_f + N_cycle S_bf
                                        + (2 N_cycle + 1) N_skip).
Integer arithmetic throughout.
"""
from __future__ import annotations


def jade_calls(P_d: int, NP: int, NG: int) -> int:
    return P_d * NP * (1 + NG)


def ens_calls(P_d: int, NP_f: int, NG_f: int, NP_bf: int, NG_bf: int, N_skip: int,
              N_cycle: int) -> int:
    S_f = NP_f * (1 + NG_f)
    S_bf = 2 * (NP_bf * (1 + NG_bf) - 1)
    est = -(-P_d // (N_skip + 1))
    return est * (S_f + N_cycle * S_bf + (2 * N_cycle + 1) * N_skip)


def search_calls(n_dom: int, NP: int, NG: int, n_imports: int, polish_steps: int) -> int:
    """Calls made by the search run here: JADE's count over n_dom samples,
    plus one call per imported individual, plus polish_steps gradient calls
    and one final call per domain when polishing."""
    polish = n_dom * (polish_steps + 1) if polish_steps > 0 else 0
    return jade_calls(n_dom, NP, NG) + n_imports + polish
