"""Philox-4x32-10 counter-based generator, vectorised over numpy arrays.

Written from the published definition: J. K. Salmon, M. A. Moraes, R. O. Dror,
D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Section 5
(the Philox S-box: two 32x32->64 multiplies per round, a Weyl key schedule,
ten rounds for the 4x32 variant).

This module holds no arithmetic of the simulated economy: it only turns
(counter, key) pairs into 32-bit words.  It is shared by the test harness
(which feeds the CPU oracle) and by anyone who wants to reproduce the
counter->draw mapping documented in ``include/econojax.h``.
"""
from __future__ import annotations

import numpy as np

# Round multipliers and Weyl key increments of Philox-4x32 (SC'11, Table 2).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3) and key (k0, k1).

    All arguments broadcast against each other; outputs are uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = (x.astype(np.uint32, copy=True) for x in (c0, c1, c2, c3))
    k0 = k0.astype(np.uint32, copy=True)
    k1 = k1.astype(np.uint32, copy=True)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            p0 = PHILOX_M0 * c0.astype(np.uint64)
            p1 = PHILOX_M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def seed_key(seed: int):
    """Split a 64-bit seed into the two 32-bit key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32)


def u01(x):
    """Map 32-bit words to float32 in [0, 1): the top 24 bits times 2**-24 (exact)."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)


def below(x, n):
    """Map 32-bit words to integers in [0, n): floor(x * n / 2**32) (Lemire's multiply-shift)."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x * np.uint64(n)) >> np.uint64(32)).astype(np.int32)
