"""Counter -> draw mapping of the synthetic workloads.

Key = the 64-bit seed (low word first).  Counters (c0, c1, c2, c3):

* population agent i of environment e at global step g (steps since
  env_reset, counting across automatic resets):
  ``(i, e, g, STREAM_POP)`` -> x0: uniform action  floor(x0 * nA / 2**32),
  x1: gather draw u in [0, 1), x2: tie-break key, x3: policy-sampling u.
* government of environment e at global step g: ``(0, e, g, STREAM_GOV)``
  -> x_b: rate level of bracket b, floor(x_b * levels / 2**32), or the
  policy-sampling uniform of bracket b.
* skills of agent i in environment e for episode k:
  ``(i, e, k, STREAM_SKILL | chunk << 8)``; the uniforms of consecutive
  chunks, in order, give SG[0..R-1] then SC (init 0, U[0, 1)); with init 1
  skill j (SG[0..R-1], then SC) is the float32 sum, in order, of the 12
  uniforms of chunks 3j, 3j+1, 3j+2, minus 5, clamped to [0, skill_max]
  (mean 1, variance 1: the distribution around 1.0 with standard deviation
  1.0 of Section 5, as an Irwin-Hall sum).

Uniforms are the top 24 bits of a word times 2**-24 (exact float32).
"""
from __future__ import annotations

import numpy as np

from .philox import below, philox4x32_10, seed_key, u01

STREAM_POP = 0
STREAM_GOV = 1
STREAM_SKILL = 2


def pop_draws(seed, env_ids, n_agents, g0, n_steps, n_actions):
    """Population draws for envs ``env_ids`` over global steps g0 .. g0+n-1.

    Returns act [n, E, A] int32, gather_u [n, E, A] float32, tb [n, E, A]
    uint32, policy_u [n, E, A] float32.  ``n_actions`` may be an int or a
    per-env array.
    """
    k0, k1 = seed_key(seed)
    env_ids = np.asarray(env_ids, dtype=np.uint32)
    g = (np.uint64(g0) + np.arange(n_steps, dtype=np.uint64)).astype(np.uint32)
    i = np.arange(n_agents, dtype=np.uint32)
    c0 = i[None, None, :]
    c1 = env_ids[None, :, None]
    c2 = g[:, None, None]
    x0, x1, x2, x3 = philox4x32_10(c0, c1, c2, np.uint32(STREAM_POP), k0, k1)
    nA = np.asarray(n_actions, dtype=np.uint64)
    if nA.ndim == 1:
        nA = nA[None, :, None]
    act = ((x0.astype(np.uint64) * nA) >> np.uint64(32)).astype(np.int32)
    return act, u01(x1), x2.astype(np.uint32), u01(x3)


def gov_draws(seed, env_ids, g0, n_steps, nb, levels):
    """Government draws: (levels [n, E, nb] int32, uniforms [n, E, nb] float32)."""
    k0, k1 = seed_key(seed)
    env_ids = np.asarray(env_ids, dtype=np.uint32)
    g = (np.uint64(g0) + np.arange(n_steps, dtype=np.uint64)).astype(np.uint32)
    xs = philox4x32_10(np.uint32(0), env_ids[None, :], g[:, None], np.uint32(STREAM_GOV), k0, k1)
    if nb > 4:
        raise ValueError("at most 4 brackets draw from one counter")
    x = np.stack(xs[:nb], axis=-1)
    return below(x, levels), u01(x)


def skill_draws(seed, env_ids, n_agents, episode, R, init=0, skill_max=5.0):
    """Skills for one episode: sg [E, A, R] float32, sc [E, A] float32."""
    k0, k1 = seed_key(seed)
    env_ids = np.asarray(env_ids, dtype=np.uint32)
    i = np.arange(n_agents, dtype=np.uint32)
    if init == 1:
        out = []
        for j in range(R + 1):
            acc = np.zeros((len(env_ids), n_agents), np.float32)
            for c in range(3):
                xs = philox4x32_10(i[None, :], env_ids[:, None], np.uint32(episode),
                                   np.uint32(STREAM_SKILL | ((3 * j + c) << 8)), k0, k1)
                for x in xs:
                    acc = (acc + u01(x).astype(np.float32)).astype(np.float32)
            out.append(np.clip((acc - np.float32(5.0)).astype(np.float32), np.float32(0.0),
                               np.float32(skill_max)).astype(np.float32))
        u = np.stack(out, axis=-1)
        return u[..., :R], u[..., R]
    n_chunks = (R + 1 + 3) // 4
    us = []
    for ch in range(n_chunks):
        xs = philox4x32_10(i[None, :], env_ids[:, None], np.uint32(episode),
                           np.uint32(STREAM_SKILL | (ch << 8)), k0, k1)
        us.extend(u01(x) for x in xs)
    u = np.stack(us, axis=-1)
    return u[..., :R].astype(np.float32), u[..., R].astype(np.float32)


def episode_inputs(seed, env_ids, A, R, nb, n_actions, levels, n_steps, T_ep, g0=0, skill_init=0,
                   skill_max=5.0):
    """Everything one oracle run needs for envs ``env_ids`` from global step g0.

    Returns a dict with act/gather_u/tb [n, E, A], gov_act [n, E, nb],
    sg0/sc0 (skills of the episode running at g0) and later_sg/later_sc
    ([k, E, A, R] / [k, E, A]) for the episodes that start during the run.
    """
    act, gu, tb, pu = pop_draws(seed, env_ids, A, g0, n_steps, n_actions)
    gov, gov_u = gov_draws(seed, env_ids, g0, n_steps, nb, levels)
    ep0 = g0 // T_ep
    sg0, sc0 = skill_draws(seed, env_ids, A, ep0, R, skill_init, skill_max)
    n_later = (g0 + n_steps) // T_ep - ep0
    later = [skill_draws(seed, env_ids, A, ep0 + 1 + k, R, skill_init, skill_max) for k in range(max(n_later, 0))]
    if later:
        later_sg = np.stack([s for s, _ in later])
        later_sc = np.stack([c for _, c in later])
    else:
        later_sg = np.zeros((0, len(np.atleast_1d(env_ids)), A, R), np.float32)
        later_sc = np.zeros((0, len(np.atleast_1d(env_ids)), A), np.float32)
    return dict(act=act, gather_u=gu, tb=tb, policy_u=pu, gov_act=gov, gov_u=gov_u,
                sg0=sg0, sc0=sc0, later_sg=later_sg, later_sc=later_sc)
