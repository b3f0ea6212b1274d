"""Uneven populations and action-space sizes in one captured rollout."""
import numpy as np
import pytest

import synth
from oracle.env import OracleEnv, default_params
from tests.parity import compare_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128
POPS = [10, 50, 37, 100, 5, 70, 10]
LEVELS = [5, 10, 20, 5, 10, 20, 20]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _weights(seed):
    import paper_2410_22165_gb300 as P
    w = {}
    for L in sorted(set(LEVELS)):
        env = P.VecEnv(1, 10, **P.price_grid(L))
        w[("pop", L)] = torch.from_numpy(synth.net_weights(seed + L, 0, env.D, H, env.nA))
        w[("gov",)] = torch.from_numpy(synth.net_weights(seed, 1, env.G, H, env.p.nb * env.p.tax_levels))
    return w


@pytest.mark.parametrize("granularity", ["exact", "by_actions"])
def test_batched_rollout_matches_oracle(granularity):
    import paper_2410_22165_gb300 as P
    T = 14
    kw = dict(T_ep=10, T_tax=4)
    br = P.BatchedRollout(POPS, LEVELS, T, _weights(3), hidden=H, precision="bf16", granularity=granularity, **kw)
    br.reset(seed=5)
    br.run()
    torch.cuda.synchronize()
    seen = set()
    for k, c in enumerate(br.classes):
        b = {n: v.cpu().numpy() for n, v in c["ro"].buf.items()}
        env = c["env"]
        p = default_params(**kw, **P.price_grid(c["P"]))
        for j, e in enumerate(c["idx"]):
            A_e = POPS[e]
            seen.add(e)
            o = OracleEnv(p, A_e)
            inp = synth.episode_inputs(5 + 7919 * k, [j], A_e, p["R"], p["nb"], o.nA, p["tax_levels"], T, p["T_ep"])
            o.reset(inp["sg0"][0], inp["sc0"][0])
            ref = o.run(b["act"][:, j, :A_e], b["gact"][:, j], inp["gather_u"][:, 0], inp["tb"][:, 0],
                        inp["later_sg"][:, 0], inp["later_sc"][:, 0])
            g = dict(rew=b["rew"][:, j], grew=b["grew"][:, j], done=b["done"][:, j], obs=b["obs"][1:, j],
                     gobs=b["gobs"][1:, j], mask=b["mask"][1:, j])
            compare_env(g, ref, env.params, A_e)
            # inactive agents of a shared-size class take no action
            assert not b["act"][:, j, A_e:].any()
    assert seen == set(range(len(POPS)))


def test_captured_graph_equals_eager():
    import paper_2410_22165_gb300 as P
    T = 6
    kw = dict(T_ep=20, T_tax=5)
    w = _weights(4)
    a = P.BatchedRollout(POPS, LEVELS, T, w, granularity="coarse", **kw)
    b = P.BatchedRollout(POPS, LEVELS, T, w, granularity="coarse", **kw)
    a.reset(seed=8)
    b.reset(seed=8)
    for _ in range(3):
        a.run()                 # eager
    b.capture()                 # one eager run inside, then the graph
    b.run()
    b.run()
    torch.cuda.synchronize()
    for ca, cb in zip(a.classes, b.classes):
        for n in ("obs", "act", "rew", "value", "logp", "done"):
            assert torch.equal(ca["ro"].buf[n], cb["ro"].buf[n]), n
        assert torch.equal(ca["env"].state, cb["env"].state)


def test_autotune_returns_a_candidate():
    import paper_2410_22165_gb300 as P
    best, rates = P.autotune(POPS, LEVELS, _weights(5), T_probe=4, repeats=1, T_ep=20, T_tax=5)
    assert best in rates and all(r > 0 for r in rates.values())


@pytest.mark.parametrize("granularity", ["exact", "coarse"])
def test_merged_policy_launches_equal_per_class_rollouts(granularity):
    """Policy launches merged across classes (one per network shape) give the
    per-class rollouts' buffers and states bit for bit, eager and captured."""
    import paper_2410_22165_gb300 as P
    T = 7
    kw = dict(T_ep=5, T_tax=3)
    w = _weights(6)
    a = P.BatchedRollout(POPS, LEVELS, T, w, granularity=granularity, merge=False, **kw)
    b = P.BatchedRollout(POPS, LEVELS, T, w, granularity=granularity, merge=True, **kw)
    # classes with the same price grid share one device copy of its weights
    assert len({c["policy"].pop_w.data_ptr() for c in b.classes}) == len(set(LEVELS))
    a.reset(seed=12)
    b.reset(seed=12)
    a.run()
    b.run()
    for _ in range(2):
        a.run()
    b.capture()                 # one eager run inside, then the graph
    b.run()
    torch.cuda.synchronize()
    for ca, cb in zip(a.classes, b.classes):
        for n, v in ca["ro"].buf.items():
            assert torch.equal(v, cb["ro"].buf[n]), n
        assert torch.equal(ca["env"].state, cb["env"].state)


def test_merged_chains_equal_per_class_rollouts():
    """Merged policy launches in 2 chains (every class split into two parts,
    part k of every class in chain k, chains on their own streams, interleaved
    per step): every part's buffers and state equal a stand-alone rollout of
    that part (the library's rollout with the same seed), eager and captured."""
    import paper_2410_22165_gb300 as P
    T = 6
    kw = dict(T_ep=5, T_tax=3)
    w = _weights(8)
    b = P.BatchedRollout(POPS, LEVELS, T, w, granularity="exact", merge=True, chains=2, **kw)
    assert {c["chain"] for c in b.classes} == {0, 1} and len(b.chain_streams) == 1
    b.reset(seed=31)
    b.capture()                 # one eager run inside, then the graph
    b.run()
    torch.cuda.synchronize()
    for k, c in enumerate(b.classes):
        env = P.VecEnv(len(c["idx"]), c["A_max"], **P.price_grid(c["P"]), **kw)
        pol = P.Policy(env, c["policy"].pop_w, c["policy"].gov_w, hidden=128, precision="bf16")
        ro = P.Rollout(env, pol, T)
        ro.reset(seed=31 + 7919 * k, pop_sizes=c["pop"])
        for r in range(2):
            if r:
                ro.carry_over()
            ro.run()
        ro.carry_over()
        torch.cuda.synchronize()
        for n, v in ro.buf.items():
            assert torch.equal(v, c["ro"].buf[n]), (k, n)
        assert torch.equal(env.state, c["env"].state), k


def test_chains_per_class_equal_one_chain():
    """Class rollouts split into 2 and 3 chains of environments (the
    autotuner's "+chainsN" candidates) give the one-chain buffers and states
    bit for bit (environments do not interact; draws are per environment)."""
    import paper_2410_22165_gb300 as P
    T = 6
    kw = dict(T_ep=5, T_tax=3)
    w = _weights(7)
    runs = [P.BatchedRollout(POPS, LEVELS, T, w, granularity="exact", chains=c, **kw) for c in (1, 2, 3)]
    for r in runs:
        r.reset(seed=21)
        r.run()
        r.run()
    torch.cuda.synchronize()
    for other in runs[1:]:
        for ca, cb in zip(runs[0].classes, other.classes):
            for n, v in ca["ro"].buf.items():
                assert torch.equal(v, cb["ro"].buf[n]), n
            assert torch.equal(ca["env"].state, cb["env"].state)


def test_full_size_classes_match_oracle():
    """The benchmark's largest classes: 500 agents on the 20-level grid (84
    actions, three mask words, 512-thread CTAs with two observation staging
    rounds) and 250 agents on the 10-level grid (256-thread CTAs), beside a
    10-agent class; a 40-step rollout with a period end and an episode end,
    compared with the oracle environment by environment."""
    import paper_2410_22165_gb300 as P
    pops, levels = [500, 250, 500, 10], [20, 10, 20, 5]
    w = {}
    for L in sorted(set(levels)):
        env = P.VecEnv(1, 10, **P.price_grid(L))
        w[("pop", L)] = torch.from_numpy(synth.net_weights(9 + L, 0, env.D, H, env.nA))
        w[("gov",)] = torch.from_numpy(synth.net_weights(9, 1, env.G, H, env.p.nb * env.p.tax_levels))
    T = 40
    kw = dict(T_ep=30, T_tax=7)
    br = P.BatchedRollout(pops, levels, T, w, hidden=H, precision="bf16", granularity="exact", **kw)
    br.reset(seed=8)
    br.run()
    torch.cuda.synchronize()
    for k, c in enumerate(br.classes):
        b = {n: v.cpu().numpy() for n, v in c["ro"].buf.items()}
        p = default_params(**kw, **P.price_grid(c["P"]))
        for j, e in enumerate(c["idx"]):
            A_e = pops[e]
            o = OracleEnv(p, A_e)
            inp = synth.episode_inputs(8 + 7919 * k, [j], A_e, p["R"], p["nb"], o.nA, p["tax_levels"], T, p["T_ep"])
            o.reset(inp["sg0"][0], inp["sc0"][0])
            ref = o.run(b["act"][:, j, :A_e], b["gact"][:, j], inp["gather_u"][:, 0], inp["tb"][:, 0],
                        inp["later_sg"][:, 0], inp["later_sc"][:, 0])
            g = dict(rew=b["rew"][:, j], grew=b["grew"][:, j], done=b["done"][:, j], obs=b["obs"][1:, j],
                     gobs=b["gobs"][1:, j], mask=b["mask"][1:, j])
            compare_env(g, ref, c["env"].params, A_e)
            assert ref["done"].sum() == 1
    assert {c["A_max"] for c in br.classes} == {10, 250, 500}
