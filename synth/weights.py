"""Seeded initial weights of the actor/critic networks.

Layout (the library's documented parameter vector, actor then critic):
W1 [in][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O],
V1 [in][H], c1 [H], V2 [H][H], c2 [H], V3 [H], c3 [1].
Each tensor starts at a multiple of 4 floats (padding between is 0).  Each
entry is uniform in [-1/sqrt(fan_in), 1/sqrt(fan_in)) (fan_in = the layer's
input width), from Philox counters (k // 4, net, 0, STREAM_WEIGHTS), word
k % 4, for flat index k of the padded vector.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10, seed_key, u01

STREAM_WEIGHTS = 3


def net_layout(in_dim, H, O):
    """[(name, shape, fan_in)] in vector order."""
    return [("W1", (in_dim, H), in_dim), ("b1", (H,), in_dim), ("W2", (H, H), H), ("b2", (H,), H),
            ("W3", (H, O), H), ("b3", (O,), H), ("V1", (in_dim, H), in_dim), ("c1", (H,), in_dim),
            ("V2", (H, H), H), ("c2", (H,), H), ("V3", (H, 1), H), ("c3", (1,), H)]


def net_offsets(in_dim, H, O):
    """[(name, shape, fan_in, offset)] and the padded length."""
    out, p = [], 0
    for name, shape, fan in net_layout(in_dim, H, O):
        out.append((name, shape, fan, p))
        p = (p + int(np.prod(shape)) + 3) // 4 * 4
    return out, p


def net_weights(seed, net_id, in_dim, H, O):
    layout, n = net_offsets(in_dim, H, O)
    k = np.arange(n, dtype=np.uint64)
    k0, k1 = seed_key(seed)
    xs = philox4x32_10((k // np.uint64(4)).astype(np.uint32), np.uint32(net_id), np.uint32(0),
                       np.uint32(STREAM_WEIGHTS), k0, k1)
    x = np.choose((k % np.uint64(4)).astype(np.int64), xs)
    u = u01(x).astype(np.float64)
    vec = np.zeros(n, np.float32)
    for _, shape, fan, off in layout:
        m = int(np.prod(shape))
        vec[off:off + m] = ((2.0 * u[off:off + m] - 1.0) / np.sqrt(fan)).astype(np.float32)
    return vec


def unpack(vec, in_dim, H, O, dtype=np.float64):
    """Flat vector -> dict of arrays (named as in the layout)."""
    layout, _ = net_offsets(in_dim, H, O)
    return {name: np.asarray(vec[off:off + int(np.prod(shape))], dtype=dtype).reshape(shape)
            for name, shape, _, off in layout}


def pack(d, in_dim, H, O):
    """dict of arrays -> flat padded float32 vector."""
    layout, n = net_offsets(in_dim, H, O)
    vec = np.zeros(n, np.float32)
    for name, shape, _, off in layout:
        vec[off:off + int(np.prod(shape))] = np.asarray(d[name], np.float32).reshape(-1)
    return vec
