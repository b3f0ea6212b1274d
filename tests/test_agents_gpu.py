"""Section 5's per-agent population networks against the float64 oracle:
independent training (iPPO: an actor and a critic per agent) and CTDE /
MAPPO (an actor per agent, one critic for all), through the C ABI.

Forward: each agent's rows against mlp64 with that agent's weights, within
the float32 bound of test_policy_gpu (chains of three dot products);
sampled actions bit-exact against the oracle's float32 sampler on the
kernel's logits.  Gradient: every parameter tensor of every agent against
ppo_loss_grad64 on that agent's minibatch rows (for a shared critic, the
mean of the agents' critic gradients, as its loss is the mean over all
rows), within 1e-3 of the tensor's largest entry (test_ppo_gpu's bound).
"""
import numpy as np
import pytest

import synth
from synth import shuffle
from oracle import policy as op
from oracle import ppo as oppo
from tests.test_policy_gpu import _check_forward

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128
ACTOR = ("W1", "b1", "W2", "b2", "W3", "b3")
CRITIC = ("V1", "c1", "V2", "c2", "V3", "c3")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _agent_weights(seed, A, D, O, hidden=H):
    """A parameter vectors, agent i's drawn from counter stream 10 + i."""
    return np.concatenate([synth.net_weights(seed, 10 + i, D, hidden, O) for i in range(A)])


def _net_of(vecs, i, layout, D, O, hidden=H):
    """Agent i's actor and the critic it uses, unpacked."""
    n = synth.net_offsets(D, hidden, O)[1]
    j = i if layout == "independent" else 0
    a = synth.unpack(vecs[i * n:(i + 1) * n], D, hidden, O)
    c = synth.unpack(vecs[j * n:(j + 1) * n], D, hidden, O)
    return {**{k: a[k] for k in ACTOR}, **{k: c[k] for k in CRITIC}}


def _policy(E, A, seed, layout, steps=37, **kw):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, **kw)
    env.reset(seed=seed)
    out = env.step(steps)
    pw = _agent_weights(seed, A, env.D, env.nA)
    gw = synth.net_weights(seed, 1, env.G, H, env.p.nb * env.p.tax_levels)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H, precision="fp32", layout=layout)
    return env, pol, out, pw, gw


@pytest.mark.parametrize("layout", ["independent", "ctde"])
def test_forward_and_sampling_per_agent(layout):
    """3 environments x 70 agents: one tile per agent, 3 of its 64 rows
    filled (the ragged case), agents beyond the first 64 included."""
    from paper_2410_22165_gb300 import _native as N
    E, A = 3, 70
    env, pol, out, pw, _ = _policy(E, A, 2, layout)
    obs, mask = out["obs"][-1].contiguous(), out["mask"][-1].contiguous()
    f = pol.forward(N.NET_POP, obs, mask, logits=True, entropy=True)
    lg, val = f["logits"].cpu().numpy(), f["value"].cpu().numpy()
    x = obs.cpu().numpy().reshape(E * A, env.D)
    for i in (0, 1, 37, A - 1):
        rows = np.arange(E) * A + i
        _check_forward(lg[rows], val[rows], _net_of(pw, i, layout, env.D, env.nA), x[rows], env.D)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    g = int(env.field("gstep")[0].item())
    u = synth.pop_draws(2, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)
    assert np.array_equal(f["act"].cpu().numpy()[:, 0], op.sample32(lg, valid, u))


def test_per_agent_networks_differ_from_shared_only_by_weights():
    """Every agent holding the same vector: the per-agent layouts give the
    shared network's outputs bit for bit."""
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    E, A = 4, 9
    env = P.VecEnv(E, A)
    env.reset(seed=4)
    out = env.step(21)
    obs, mask = out["obs"][-1].contiguous(), out["mask"][-1].contiguous()
    w = synth.net_weights(4, 0, env.D, H, env.nA)
    gw = torch.from_numpy(synth.net_weights(4, 1, env.G, H, env.p.nb * env.p.tax_levels))
    ref = P.Policy(env, torch.from_numpy(w), gw, hidden=H).forward(N.NET_POP, obs, mask, logits=True)
    for layout in ("independent", "ctde"):
        pol = P.Policy(env, torch.from_numpy(np.tile(w, A)), gw, hidden=H, layout=layout)
        got = pol.forward(N.NET_POP, obs, mask, logits=True)
        for k in ("logits", "value", "act", "logp"):
            assert torch.equal(got[k], ref[k]), (layout, k)


@pytest.mark.parametrize("layout", ["independent", "ctde"])
def test_minibatch_gradient_per_agent(layout):
    """4 environments x 3 agents x 16 steps, 4 minibatches of the 64 (step,
    environment) positions: minibatch 1 of shuffle 3 for every agent."""
    import paper_2410_22165_gb300 as P
    E, A, T = 4, 3, 16
    env, pol, _, pw, gw = _policy(E, A, 6, layout, T_ep=12, T_tax=4)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=6)
    ro.run()
    ppo = P.PPO(pol, T, minibatches=4, seed=77)
    ppo.advantages(ro)
    grad, stats = ppo.minibatch_grad(ro, 0, 3, 1)
    grad = grad.cpu().numpy()
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    pp = ppo.pp
    done = np.repeat(b["done"][:, :, None], A, axis=2).reshape(T, E * A)
    adv, ret = oppo.gae64(b["rew"].reshape(T, E * A), b["value"].reshape(T + 1, E * A), done, pp.gamma, pp.lam)
    pos = shuffle.minibatch_rows(1, 4, T * E, 77, 3)
    n = synth.net_offsets(env.D, H, env.nA)[1]
    critic_sum = None
    for i in range(A):
        rows = pos * A + i
        x = b["obs"][:T].reshape(T * E * A, env.D)[rows]
        valid = op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows]
        _, g64, _ = oppo.ppo_loss_grad64(_net_of(pw, i, layout, env.D, env.nA), x, b["act"].reshape(-1, 1)[rows],
                                         valid, b["logp"].reshape(-1)[rows], b["value"][:T].reshape(-1)[rows],
                                         adv.reshape(-1)[rows], ret.reshape(-1)[rows], clip=pp.clip,
                                         vf_coef=pp.vf_coef, vclip=pp.vclip, ent_coef=pp.ent_coef, heads=1,
                                         head=env.nA)
        got = synth.unpack(grad[i * n:(i + 1) * n], env.D, H, env.nA)
        keys = ACTOR + (CRITIC if layout == "independent" else ())
        for k in keys:
            ref = g64[k]
            assert np.max(np.abs(got[k].reshape(ref.shape) - ref)) <= 1e-3 * np.abs(ref).max() + 1e-7, (i, k)
        if layout == "ctde":
            critic_sum = {k: g64[k] / A + (critic_sum[k] if critic_sum else 0.0) for k in CRITIC}
            if i > 0:
                assert not any(got[k].any() for k in CRITIC), "unused critic parts get zero gradients"
    if layout == "ctde":
        got0 = synth.unpack(grad[:n], env.D, H, env.nA)
        for k, ref in critic_sum.items():
            assert np.max(np.abs(got0[k].reshape(ref.shape) - ref)) <= 1e-3 * np.abs(ref).max() + 1e-7, k
    assert np.isfinite(stats.cpu().numpy()).all()


@pytest.mark.parametrize("layout", ["independent", "ctde"])
def test_update_moves_every_agent(layout):
    """A whole update (2 epochs x 2 minibatches, both networks): finite,
    every agent's actor moves, a CTDE critic only in vector 0."""
    import paper_2410_22165_gb300 as P
    E, A, T = 4, 5, 12
    env, pol, _, pw, _ = _policy(E, A, 8, layout, T_ep=10, T_tax=5)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=8)
    ro.run()
    ppo = P.PPO(pol, T, epochs=2, minibatches=2, seed=3)
    before = pol.pop_w.clone()
    stats = ppo.update(ro).cpu().numpy()
    assert np.isfinite(stats).all()
    d = (pol.pop_w - before).cpu().numpy().reshape(A, -1)
    n = synth.net_offsets(env.D, H, env.nA)[1]
    for i in range(A):
        di = synth.unpack(d[i], env.D, H, env.nA)
        assert np.abs(di["W2"]).max() > 0, i
        if layout == "ctde" and i > 0:
            assert not np.abs(di["V2"]).any()
        else:
            assert np.abs(di["V2"]).max() > 0


@pytest.mark.parametrize("hidden", [128, 256])
@pytest.mark.parametrize("layout", ["independent", "ctde"])
def test_bf16_forward_per_agent(layout, hidden):
    """The tensor-core forward with per-agent weights (hidden 128: one CTA per
    tile; hidden 256: the two-CTA cluster kernel): 300 environments x 7
    agents (3 tiles per agent, the last ragged; CTAs crossing agents repack),
    each agent's rows within the BF16 bound of test_policy_gpu, sampled
    actions bit-exact against the oracle's float32 sampler on the kernel's
    logits; a BF16 rollout runs."""
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    from tests.test_policy_gpu import _bound, magnitude
    E, A = 300, 7
    env = P.VecEnv(E, A)
    env.reset(seed=3)
    out = env.step(29)
    pw = _agent_weights(3, A, env.D, env.nA, hidden)
    gw = synth.net_weights(3, 1, env.G, hidden, env.p.nb * env.p.tax_levels)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=hidden, precision="bf16", layout=layout)
    obs, mask = out["obs"][-1].contiguous(), out["mask"][-1].contiguous()
    f = pol.forward(N.NET_POP, obs, mask, logits=True)
    lg, val = f["logits"].cpu().numpy(), f["value"].cpu().numpy()
    x = obs.cpu().numpy().reshape(E * A, env.D)
    for i in range(A):
        rows = np.arange(E) * A + i
        w = _net_of(pw, i, layout, env.D, env.nA, hidden)
        lg64, v64 = op.mlp64(w, x[rows])
        mlg, mv = magnitude(w, x[rows])
        bound = _bound("bf16", env.D)
        assert np.all(np.abs(lg[rows] - lg64) <= bound * mlg + 1e-30), i
        assert np.all(np.abs(val[rows] - v64) <= bound * mv + 1e-30), i
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    g = int(env.field("gstep")[0].item())
    u = synth.pop_draws(3, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)
    assert np.array_equal(f["act"].cpu().numpy()[:, 0], op.sample32(lg, valid, u))
    ro = P.Rollout(env, pol, 5)
    ro.reset(seed=3)
    ro.run()
    torch.cuda.synchronize()
    assert torch.isfinite(ro.buf["value"]).all() and (ro.buf["act"] >= 0).all()


def test_bf16_per_agent_update_is_refused():
    """The per-agent PPO gradient is FP32 only (host check, nothing runs)."""
    import ctypes as C
    from paper_2410_22165_gb300 import _native as N
    p = N.make_params(E=2, A=4)
    pp = N.EjPpoParams()
    N.load().ej_ppo_params_default(C.byref(pp))
    fake = C.c_void_p(4096)
    b = N.EjRollout(**{f: 4096 for f, _ in N.EjRollout._fields_})
    st = N.load().ppo_minibatch_grad_agents(C.byref(p), C.byref(pp), 8, H, N.BF16, N.NETS_CTDE, fake, C.byref(b),
                                            fake, 0, 0, fake, None, None)
    assert st == 3
