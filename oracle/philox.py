"""Philox4x32-10 counter-based generator (TEST INFRASTRUCTURE).

Written from its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4 x 32-bit counter is passed through 10 rounds; each round
multiplies counter words 0 and 2 by the constants M0 = 0xD2511F53 and
M1 = 0xCD9E8D57 into 64-bit products, and returns

    (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0)),

the 2 x 32-bit key being bumped by the Weyl constants (0x9E3779B9,
0xBB67AE85) between rounds. The paper leaves its generator unspecified;
the search draws every random number from this function keyed by
(sample, generation, individual), so runs are reproducible and resumable.
Plain Python integers.
"""
from __future__ import annotations

MASK = 0xFFFFFFFF
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(v) & MASK for v in ctr)
    k0, k1 = (int(v) & MASK for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, \
                         ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return c0, c1, c2, c3


def words(seed: int, domain: int, gen: int, individual: int, n: int):
    """The first n 32-bit words drawn for (domain, gen, individual).

    key = (low, high) 32-bit halves of the 64-bit seed; the stream of words
    is philox(counter = (individual, gen, domain, s)) for s = 0, 1, ...,
    four words per block, concatenated.
    """
    key = (seed & MASK, (seed >> 32) & MASK)
    out = []
    s = 0
    while len(out) < n:
        out.extend(philox4x32_10((individual, gen, domain, s), key))
        s += 1
    return out[:n]
