"""CPU oracle of GAE and the clipped PPO update (test infrastructure only).

Section 4 trains population and government with PPO (Table 2: clip 0.2,
value-function coefficient 0.25, value clip 10, entropy coefficient 0.1,
GAE lambda 0.95); the benchmark configuration sets gamma 0.99.

* ``gae64``: generalised advantage estimation, the reverse recursion
  A_t = delta_t + gamma lambda (1 - done_t) A_{t+1},
  delta_t = r_t + gamma (1 - done_t) V_{t+1} - V_t, returns = A + V.
* ``ppo_loss_grad64``: the clipped surrogate, the clipped value loss and the
  entropy bonus of a minibatch, and their gradient with respect to every
  parameter of the actor and critic, by hand-written backpropagation in
  float64 (ReLU networks of ``policy.mlp64``).
  With ``operand=bf16_round`` every product operand is first rounded to
  bfloat16 (the BF16 tensor-core form of the update, FP32/FP64 sums).
* ``adam64``: one Adam step (Kingma and Ba, 2015).
"""
from __future__ import annotations

import numpy as np


def gae64(rew, value, done, gamma, lam):
    """rew [T, N], value [T+1, N], done [T, N] -> adv [T, N], ret [T, N]."""
    rew = np.asarray(rew, np.float64)
    value = np.asarray(value, np.float64)
    nd = 1.0 - np.asarray(done, np.float64)
    T = rew.shape[0]
    adv = np.zeros_like(rew)
    nxt = np.zeros(rew.shape[1])
    for t in range(T - 1, -1, -1):
        delta = rew[t] + gamma * nd[t] * value[t + 1] - value[t]
        nxt = delta + gamma * lam * nd[t] * nxt
        adv[t] = nxt
    return adv, adv + value[:-1]


def _heads_softmax(logits, valid, heads, head):
    """Per-head masked softmax: p, log p (0 where invalid), entropy per row."""
    N = logits.shape[0]
    p = np.zeros_like(logits)
    logp = np.zeros_like(logits)
    ent = np.zeros(N)
    for h in range(heads):
        sl = slice(h * head, (h + 1) * head)
        l = np.where(valid[:, sl], logits[:, sl], -np.inf)
        m = l.max(1, keepdims=True)
        z = np.where(valid[:, sl], np.exp(l - m), 0.0)
        S = z.sum(1, keepdims=True)
        p[:, sl] = z / S
        logp[:, sl] = np.where(valid[:, sl], l - m - np.log(S), 0.0)
        ent -= (p[:, sl] * logp[:, sl]).sum(1)
    return p, logp, ent


def bf16_round(a):
    """Nearest bfloat16 value (ties to even) of each entry, via float32: the
    rounding a BF16 GEMM operand goes through (8-bit significand)."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def ppo_loss_grad64(w, x, act, valid, logp_old, v_old, adv, ret, *, clip, vf_coef, vclip,
                    ent_coef, heads=1, head=None, normalize_adv=True, operand=None, moments=None):
    """Loss (float) and gradients (dict like w) of one minibatch.

    x [N, in], act [N, heads] int, valid [N, heads*head] bool, logp_old [N],
    v_old [N], adv [N] (raw GAE), ret [N].

    operand: applied to every matrix-product operand (weights, inputs,
    activations, backward signals) before the product; None = exact.  With
    bf16_round this is the BF16-operand form: operands rounded to bfloat16,
    products and sums in float64.

    moments: None, or (n, sum, sum of squares) of the advantages of a larger
    minibatch these rows belong to (the union over the ranks of a
    data-parallel update): advantages are normalised with its mean and
    population std and every mean is over its n rows, so the returned loss and
    gradient are these rows' part of the larger minibatch's (parts sum to the
    whole)."""
    R = operand if operand is not None else (lambda t: t)
    x = np.asarray(x, np.float64)
    N = x.shape[0]
    act = np.asarray(act).reshape(N, heads)
    if head is None:
        head = valid.shape[1] // heads
    a = np.asarray(adv, np.float64)
    if moments is not None:
        n_tot = float(moments[0])
        mu = float(moments[1]) / n_tot
        sd = np.sqrt(max(float(moments[2]) / n_tot - mu * mu, 0.0))
        if normalize_adv:
            a = (a - mu) / (sd + 1e-8)
    else:
        n_tot = float(N)
        if normalize_adv:
            a = (a - a.mean()) / (a.std() + 1e-8)
    # forward
    x = R(x)
    W1, W2, W3 = R(w["W1"]), R(w["W2"]), R(w["W3"])
    V1, V2, V3 = R(w["V1"]), R(w["V2"]), R(w["V3"])
    z1 = x @ W1 + w["b1"]; h1 = R(np.maximum(z1, 0))
    z2 = h1 @ W2 + w["b2"]; h2 = R(np.maximum(z2, 0))
    logits = h2 @ W3 + w["b3"]
    y1 = x @ V1 + w["c1"]; g1 = R(np.maximum(y1, 0))
    y2 = g1 @ V2 + w["c2"]; g2 = R(np.maximum(y2, 0))
    v = (g2 @ V3 + w["c3"])[:, 0]
    p, logp_all, ent = _heads_softmax(logits, valid, heads, head)
    logp = sum(logp_all[np.arange(N), h * head + act[:, h]] for h in range(heads))
    ratio = np.exp(logp - logp_old)
    cr = np.clip(ratio, 1 - clip, 1 + clip)
    surr = np.minimum(ratio * a, cr * a)
    vc = v_old + np.clip(v - v_old, -vclip, vclip)
    la, lb = (v - ret) ** 2, (vc - ret) ** 2
    lv = 0.5 * np.maximum(la, lb)
    loss = (-surr.sum() + vf_coef * lv.sum() - ent_coef * ent.sum()) / n_tot
    # backward: d loss / d logp, d logits, d value
    unclipped = ratio * a <= cr * a
    inside = (ratio > 1 - clip) & (ratio < 1 + clip)
    dratio = np.where(unclipped, -a, np.where(inside, -a, 0.0)) / n_tot
    dlogp = dratio * ratio
    dlog = np.zeros_like(logits)
    for h in range(heads):
        sl = slice(h * head, (h + 1) * head)
        onehot = np.zeros((N, head)); onehot[np.arange(N), act[:, h]] = 1.0
        dlog[:, sl] = dlogp[:, None] * (onehot - p[:, sl])
        Hh = -(p[:, sl] * logp_all[:, sl]).sum(1)
        dlog[:, sl] += (ent_coef / n_tot) * p[:, sl] * (logp_all[:, sl] + Hh[:, None])
    dlog = np.where(valid, dlog, 0.0)
    dv = np.where(la >= lb, v - ret, (vc - ret) * (np.abs(v - v_old) < vclip)) * (vf_coef / n_tot)
    g = {}
    dlog = R(dlog)
    g["W3"] = h2.T @ dlog; g["b3"] = dlog.sum(0)
    dz2 = R((dlog @ W3.T) * (z2 > 0))
    g["W2"] = h1.T @ dz2; g["b2"] = dz2.sum(0)
    dz1 = R((dz2 @ W2.T) * (z1 > 0))
    g["W1"] = x.T @ dz1; g["b1"] = dz1.sum(0)
    dvv = dv[:, None]
    g["V3"] = g2.T @ R(dvv); g["c3"] = R(dvv).sum(0)
    dy2 = R((dvv @ w["V3"].T) * (y2 > 0))      # a rank-1 product, formed before rounding
    g["V2"] = g1.T @ dy2; g["c2"] = dy2.sum(0)
    dy1 = R((dy2 @ V2.T) * (y1 > 0))
    g["V1"] = x.T @ dy1; g["c1"] = dy1.sum(0)
    stats = dict(loss=loss, pg=-surr.mean(), vf=lv.mean(), ent=ent.mean(),
                 clipfrac=float(np.mean(np.abs(ratio - 1) > clip)))
    return loss, g, stats


def adam64(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-5):
    """One Adam step (step counts from 1); returns new (param, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v
