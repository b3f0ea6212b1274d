"""Comparison of the CUDA environment with the CPU oracle.

Tolerances (float outputs; integer state and masks are compared exactly):
  * observations, statistics: |gpu - oracle| <= 1e-5 * max(|scale|, 1), where
    the scale is the value itself (observation features: period earnings,
    coin in escrow and all others), for liquid coin the largest coin the
    agent has held since its episode began (a float sum keeps the absolute
    error of the largest value it passed; the coin contract's reading of
    "relative"), the largest of mean / std / median of the same metric
    (government statistics), or the utility magnitude of the agent at this or
    the previous step (rewards: the difference of two utilities loses the
    relative precision of each);
  * government reward: 1e-5 * max(total coin, 1).
The float "decision mirror" of the oracle must equal the GPU's liquid coin
bit for bit.
"""
from __future__ import annotations

import numpy as np

import synth
from oracle.env import OracleEnv

REL = 1e-5


def oracle_run(params, A_e, e, seed, T, g0=0):
    o = OracleEnv(params, A_e)
    inp = synth.episode_inputs(seed, [e], A_e, params["R"], params["nb"], o.nA,
                               params["tax_levels"], T, params["T_ep"], g0=g0,
                               skill_init=params.get("skill_init", 0), skill_max=params.get("skill_max", 5.0))
    o.reset(inp["sg0"][0], inp["sc0"][0])
    out = o.run(inp["act"][:, 0], inp["gov_act"][:, 0], inp["gather_u"][:, 0], inp["tb"][:, 0],
                inp["later_sg"][:, 0], inp["later_sc"][:, 0])
    return o, out


def _close(g, o, scale, what):
    g = np.asarray(g, np.float64)
    bound = REL * np.maximum(np.abs(scale), 1.0)
    err = np.abs(g - o)
    bad = err > bound
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} values out of tolerance, first at {idx.tolist()}: "
                             f"gpu={g[tuple(idx[0])]} oracle={o[tuple(idx[0])]} bound={bound[tuple(idx[0])]}")
    return float((err / np.maximum(np.abs(scale), 1.0)).max()) if err.size else 0.0


def coin_scale(coin, done, start_coin):
    """[n, A]: the largest |coin| each agent has held since its episode began
    (start coin included), step by step; done[s] = 1 means row s is already
    the first state of the next episode."""
    n, A = coin.shape
    out = np.empty_like(coin, dtype=np.float64)
    run = np.full(A, abs(float(start_coin)))
    for s in range(n):
        if done[s]:
            run = np.full(A, abs(float(start_coin)))
        run = np.maximum(run, np.abs(coin[s]))
        out[s] = run
    return out


def compare_env(g, ref, params, A_e, obs0_ref=None):
    """g: GPU outputs of one env as numpy (rew [n,A], grew [n], done [n], obs [n,A,D],
    gobs [n,G], mask [n,A,W]); ref: oracle outputs (A_e agents).  Returns max rel errors."""
    R, eta = params["R"], params["eta"]
    errs = {}
    if "done" in g:
        assert np.array_equal(g["done"].astype(np.int32), ref["done"]), "done differs"
    if "mask" in g:
        m = g["mask"].view(np.uint32)
        assert np.array_equal(m[:, :A_e], ref["mask"]), "mask differs"
        assert not m[:, A_e:].any(), "mask of absent agents not zero"
    if "obs" in g:
        go, ro = g["obs"], ref["obs"]
        ints = list(range(3, 3 + 2 * R))
        assert np.array_equal(go[:, :A_e, ints].astype(np.int64), ro[:, :, ints].astype(np.int64)), \
            "integer observation features (inventories) differ"
        scale = np.abs(ro).copy()
        done = ref["done"] if "done" in ref else np.zeros(len(ro), bool)
        scale[:, :, 0] = coin_scale(ro[:, :, 0], done, params["start_coin"])
        errs["obs"] = _close(go[:, :A_e], ro, scale, "obs")
        D = ro.shape[2]
        rel = lambda f, sc: float((np.abs(go[:, :A_e, f] - ro[:, :, f]) / np.maximum(sc, 1.0)).max())
        errs["coin"] = rel(0, scale[:, :, 0])
        errs["coin_plain"] = rel(0, np.abs(ro[:, :, 0]))
        errs["earnings"] = rel(D - 3, np.abs(ro[:, :, D - 3]))
        assert not go[:, A_e:].any(), "obs of absent agents not zero"
    if "rew" in g:
        ro = ref["obs"]
        C = ro[:, :, 0] + ro[:, :, 1]
        u = np.abs(np.power(C, 1 - eta) / (1 - eta)) + ro[:, :, 2] + 1.0
        prev = np.concatenate([u[:1] if obs0_ref is None else
                               (np.abs(np.power(obs0_ref[:, 0] + obs0_ref[:, 1], 1 - eta) / (1 - eta))
                                + obs0_ref[:, 2] + 1.0)[None], u[:-1]])
        scale = np.maximum(u, prev)
        # a reward is the difference of two utilities: its error is bounded by the
        # sum of their magnitudes (at an episode end the earlier one stands for both)
        errs["rew"] = _close(g["rew"][:, :A_e], ref["rew"], scale * 2, "rew")
        assert not g["rew"][:, A_e:].any()
    if "gobs" in g:
        M = 3
        ro = ref["gobs"]
        scale = np.zeros_like(ro)
        for m in range(M):
            s = np.max(np.abs(ro[:, 3 * m:3 * m + 3]), axis=1, keepdims=True)
            scale[:, 3 * m:3 * m + 3] = s
        scale[:, 3 * M:] = np.abs(ro[:, 3 * M:])
        errs["gobs"] = _close(g["gobs"], ro, scale, "gobs")
    if "grew" in g:
        prod = ref["gobs"][:, 0] * A_e
        scale = np.maximum(prod, np.concatenate([prod[:1], prod[:-1]])) * 2
        errs["grew"] = _close(g["grew"], ref["grew"], scale, "grew")
    return errs
