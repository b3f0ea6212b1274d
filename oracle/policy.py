"""CPU oracle of the policy side of the hot path (test infrastructure only).

* ``mlp64``: the actor and critic MLPs of Section 4 ("two layers with 128
  nodes", shared by all population agents; ReLU hidden activations, the
  activation the benchmark configuration names) in float64, one layer at a
  time with numpy matmul as the only primitive.
* ``exp32``: exp in float32 by Cody-Waite argument reduction (W. J. Cody and
  W. Waite, "Software Manual for the Elementary Functions", 1980: x = n ln2 + r
  with ln2 split into a short high part and a low part) and the degree-7
  Taylor polynomial of e^r on |r| <= ln2/2, evaluated by Horner's rule, one
  float32 rounding per operation.  The CUDA sampler uses the same published
  method, so a sampled action (an integer decided by float arithmetic) is
  decided in the same precision by the same steps on both sides.
* ``sample32``: masked categorical sampling (Section 3 "Action masking":
  forbidden actions get probability zero) by inverse CDF on float32.
* ``logp_entropy64``: log-probability and entropy of a masked softmax in
  float64.
"""
from __future__ import annotations

import numpy as np

F = np.float32
LOG2E = F(1.44269504)
LN2_HI = F(0.693145751953125)       # 0x3F317200: few significant bits, n * LN2_HI exact
LN2_LO = F(1.42860677e-06)
EXP_CUTOFF = F(-80.0)               # below: 0 (e^-80 ~ 1.8e-35)
TAYLOR = [F(1.0 / 5040.0), F(1.0 / 720.0), F(1.0 / 120.0), F(1.0 / 24.0), F(1.0 / 6.0), F(0.5), F(1.0), F(1.0)]


def exp32(x):
    """e^x in float32 for x <= 0 (Cody-Waite + degree-7 Taylor)."""
    x = np.asarray(x, dtype=F)
    n = np.rint(x * LOG2E).astype(F)
    r = (x - n * LN2_HI).astype(F)
    r = (r - n * LN2_LO).astype(F)
    p = np.full_like(r, TAYLOR[0])
    for c in TAYLOR[1:]:
        p = (p * r).astype(F)
        p = (p + c).astype(F)
    ni = np.clip(n, -126, 127).astype(np.int32)
    scale = ((ni + 127).astype(np.uint32) << np.uint32(23)).view(F)
    out = (p * scale).astype(F)
    return np.where(x < EXP_CUTOFF, F(0.0), out).astype(F)


def mask_bits(mask_words, n_actions):
    """[..., W] uint32 words -> [..., n_actions] bool."""
    m = np.asarray(mask_words, dtype=np.uint32)
    a = np.arange(n_actions)
    return ((m[..., a // 32] >> (a % 32).astype(np.uint32)) & 1).astype(bool)


def sample32(logits, valid, u):
    """Inverse-CDF draw from the masked softmax of float32 logits.

    logits [N, K] float32, valid [N, K] bool, u [N] float32 in [0, 1).
    Weights w_j = exp32(l_j - max valid l), summed in action order; the action
    is the first valid j whose running sum exceeds u * sum (the last valid
    action if rounding leaves none)."""
    logits = np.asarray(logits, dtype=F)
    N, K = logits.shape
    neg = np.where(valid, logits, -np.inf).astype(F)
    m = neg.max(axis=1)
    m = np.where(np.isfinite(m), m, F(0.0)).astype(F)
    w = np.where(valid, exp32((logits - m[:, None]).astype(F)), F(0.0)).astype(F)
    S = np.zeros(N, F)
    for j in range(K):
        S = (S + w[:, j]).astype(F)
    thr = (np.asarray(u, F) * S).astype(F)
    act = np.full(N, -1, np.int64)
    last_valid = np.where(valid.any(1), K - 1 - np.argmax(valid[:, ::-1], axis=1), 0)
    c = np.zeros(N, F)
    for j in range(K):
        c = np.where(valid[:, j], (c + w[:, j]).astype(F), c).astype(F)
        hit = (act < 0) & valid[:, j] & (c > thr)
        act[hit] = j
    act[act < 0] = last_valid[act < 0]
    return act.astype(np.int32)


def logp_entropy64(logits, valid, act):
    l = np.asarray(logits, dtype=np.float64)
    l = np.where(valid, l, -np.inf)
    m = l.max(axis=1, keepdims=True)
    z = np.exp(l - m)
    S = z.sum(axis=1, keepdims=True)
    logp_all = l - m - np.log(S)
    p = z / S
    ent = -np.where(valid, p * np.where(valid, logp_all, 0.0), 0.0).sum(1)
    logp = np.take_along_axis(logp_all, np.asarray(act)[:, None].astype(np.int64), 1)[:, 0]
    return logp, ent


def relu(x):
    return np.maximum(x, 0.0)


def mlp64(w, x):
    """Actor logits and critic value of Section 4's 2 x 128 networks, float64.

    w: dict of float64 arrays W1 [in,H], b1, W2 [H,H], b2, W3 [H,O], b3,
    V1 [in,H], c1, V2 [H,H], c2, V3 [H,1], c3."""
    x = np.asarray(x, dtype=np.float64)
    h = relu(x @ w["W1"] + w["b1"])
    h = relu(h @ w["W2"] + w["b2"])
    logits = h @ w["W3"] + w["b3"]
    g = relu(x @ w["V1"] + w["c1"])
    g = relu(g @ w["V2"] + w["c2"])
    value = (g @ w["V3"] + w["c3"])[:, 0]
    return logits, value
