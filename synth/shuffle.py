"""Seeded minibatch shuffles: a random permutation of [0, N) computed per index.

A Feistel network (Luby and Rackoff, "How to construct pseudorandom
permutations from pseudorandom functions", SIAM J. Comput. 1988) on b bits,
2^b the smallest power of two >= N (b >= 2), with 4 rounds is a permutation of
[0, 2^b); walking the cycle until the value falls below N (Black and Rogaway,
"Ciphers with arbitrary finite domains", CT-RSA 2002) restricts it to a
permutation of [0, N).  Alternating (unbalanced) form: the high part has
floor(b/2) bits, the low part the rest; each round XORs the part that is not
its input with the round function of the other part (masked to the replaced
part's width) and swaps the two, so the widths are back in place after the
four rounds; with b even it is the balanced network.  The round function is
Philox word x0 at counter (part, round, epoch_counter, STREAM_SHUFFLE) under
the seed key.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10, seed_key

STREAM_SHUFFLE = 4


def domain_bits(N):
    b = 2
    while (1 << b) < N:
        b += 1
    return b


def feistel(x, bits, seed, ctr):
    k0, k1 = seed_key(seed)
    wa = bits // 2
    wb = bits - wa
    A = x >> np.uint32(wb)
    B = x & np.uint32((1 << wb) - 1)
    la, lb = wa, wb
    for rnd in range(4):
        m = np.uint32((1 << la) - 1)
        F = philox4x32_10(B, np.uint32(rnd), np.uint32(ctr), np.uint32(STREAM_SHUFFLE), k0, k1)[0] & m
        A, B = B, (A ^ F) & m
        la, lb = lb, la
    return (A << np.uint32(wb)) | B


def permute(idx, N, seed, ctr):
    """pi(idx) for the permutation of [0, N) keyed by (seed, ctr)."""
    bits = domain_bits(N)
    x = feistel(np.asarray(idx, np.uint32), bits, seed, ctr)
    bad = x >= N
    while bad.any():
        x[bad] = feistel(x[bad], bits, seed, ctr)
        bad = x >= N
    return x.astype(np.int64)


def minibatch_rows(m, n_minibatches, N, seed, ctr):
    """Rows of minibatch m: pi(p) for positions p in [floor(mN/M), floor((m+1)N/M))."""
    lo, hi = (m * N) // n_minibatches, ((m + 1) * N) // n_minibatches
    return permute(np.arange(lo, hi, dtype=np.uint32), N, seed, ctr)
