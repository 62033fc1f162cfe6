"""CPU oracle for the traveltime-parameter search (TEST INFRASTRUCTURE).

A plain, slow, obviously-correct restatement of what the GPU path computes,
written from the paper (Ultra-fast traveltime parameters search by a
coevolutionary optimization approach using GPUs, arXiv 2304.11399) and the
textbook definitions it cites. It shares no code with the CUDA library and
imports nothing from it. Only the test-suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference leg may import it; the product
path never calls it and has no CPU fallback.

Modules
-------
semblance  FP64 traveltime operators (CMP, ZO-CRS), windowed linear
           interpolation, Neidell-Taner semblance and its analytic gradient.
philox     Philox4x32-10 counter-based generator (Salmon et al., SC'11).
de         One differential-evolution generation (init, selection, best,
           DE/current-to-best/1/bin mutation+crossover, bound repair) in FP32,
           the precision the search's integer decisions are taken in.
jade       JADE's adaptation of F and CR (normal / Cauchy draws around a
           memory updated from successful children) and its archive of
           replaced parents, with only correctly rounded float32 operations.
exchange   Neighbour exchange of best individuals between adjacent domains.
search     The whole search (DE + exchange + gradient polish).
ens        Evolution by neighborhood similarity in sweep mode (forward
           exploration, backward-and-forward cycles, N_skip interpolation).
stack      Stacked zero-offset output along an operator (mean centre
           amplitude over the aperture).
counts     Semblance-call counts of JADE (eq. jade_semblance) and ENS
           (eq. ens_semblance).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, hand-worked fixtures, known-answer vectors, brute force,
finite differences); none is "parity unpinned".
"""
from . import semblance, philox, de, jade, exchange, search, counts, ens, stack  # noqa: F401
