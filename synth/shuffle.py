"""Seeded minibatch shuffles: a random permutation of [0, N) computed per index.

A balanced Feistel network (Luby and Rackoff, "How to construct pseudorandom
permutations from pseudorandom functions", SIAM J. Comput. 1988) on 2h bits
with 4 rounds is a permutation of [0, 4^h); walking the cycle until the value
falls below N (Black and Rogaway, "Ciphers with arbitrary finite domains",
CT-RSA 2002) restricts it to a permutation of [0, N).  The round function is
the low h bits of Philox word x0 at counter (R, round, epoch_counter,
STREAM_SHUFFLE) under the seed key.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10, seed_key

STREAM_SHUFFLE = 4


def half_bits(N):
    b = max(2, int(np.ceil(np.log2(max(N, 2)))))
    b += b & 1
    return b // 2


def feistel(x, half, seed, ctr):
    k0, k1 = seed_key(seed)
    mask = np.uint32((1 << half) - 1)
    L = (x >> np.uint32(half)) & mask
    R = x & mask
    for rnd in range(4):
        F = philox4x32_10(R, np.uint32(rnd), np.uint32(ctr), np.uint32(STREAM_SHUFFLE), k0, k1)[0] & mask
        L, R = R, (L ^ F) & mask
    return (L << np.uint32(half)) | R


def permute(idx, N, seed, ctr):
    """pi(idx) for the permutation of [0, N) keyed by (seed, ctr)."""
    half = half_bits(N)
    x = feistel(np.asarray(idx, np.uint32), half, seed, ctr)
    bad = x >= N
    while bad.any():
        x[bad] = feistel(x[bad], half, seed, ctr)
        bad = x >= N
    return x.astype(np.int64)


def minibatch_rows(m, n_minibatches, N, seed, ctr):
    """Rows of minibatch m: pi(p) for positions p in [floor(mN/M), floor((m+1)N/M))."""
    lo, hi = (m * N) // n_minibatches, ((m + 1) * N) // n_minibatches
    return permute(np.arange(lo, hi, dtype=np.uint32), N, seed, ctr)
