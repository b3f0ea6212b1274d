"""Parity of GAE, the PPO minibatch gradient and the update with the float64
oracle, on small slices (2-8 environments x 4-7 agents).

Gradient tolerance: every entry is a sum over minibatch rows of products
formed through three float32 dot products (K <= 128) and float32 exp/log;
entries are compared to the float64 gradient within 1e-3 of the largest
entry of the same tensor.
"""
import numpy as np
import pytest

import synth
from synth import shuffle
from oracle import ppo as oppo
from oracle import policy as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _setup(E, A, T, seed=0, ppo_kw=None, **kw):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, **kw)
    O_gov = env.p.nb * env.p.tax_levels
    pw = synth.net_weights(seed, 0, env.D, H, env.nA)
    gw = synth.net_weights(seed, 1, env.G, H, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=seed)
    ro.run()
    ppo = P.PPO(pol, T, **(ppo_kw or {}))
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    return env, pol, ro, ppo, b, pw, gw


def _oracle_gae(env, b, pp):
    E, A = env.E, env.A
    T = b["rew"].shape[0]
    done = np.repeat(b["done"][:, :, None], A, axis=2).reshape(T, E * A)
    adv, ret = oppo.gae64(b["rew"].reshape(T, E * A), b["value"].reshape(T + 1, E * A), done, pp.gamma, pp.lam)
    gadv, gret = oppo.gae64(b["grew"], b["gvalue"], b["done"], pp.gamma, pp.lam)
    return adv, ret, gadv, gret


def test_gae_matches_oracle():
    env, pol, ro, ppo, b, *_ = _setup(3, 7, 24, seed=1, T_ep=10, T_tax=5)
    g = {k: v.cpu().numpy() for k, v in ppo.advantages(ro).items()}
    adv, ret, gadv, gret = _oracle_gae(env, b, ppo.pp)
    T = 24
    for got, ref in ((g["adv"].reshape(T, -1), adv), (g["ret"].reshape(T, -1), ret),
                     (g["gadv"], gadv), (g["gret"], gret)):
        scale = np.abs(ref).max() + 1.0
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale * T


def _oracle_grad(env, b, pp, net, rows, adv, ret, wvec):
    E, A = env.E, env.A
    T = b["rew"].shape[0]
    if net == 0:
        x = b["obs"][:T].reshape(T * E * A, env.D)[rows]
        valid = op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows]
        act = b["act"].reshape(-1, 1)[rows]
        lpo = b["logp"].reshape(-1)[rows]
        vo = b["value"][:T].reshape(-1)[rows]
        a, r = adv.reshape(-1)[rows], ret.reshape(-1)[rows]
        w = synth.unpack(wvec, env.D, H, env.nA)
        heads, head = 1, env.nA
    else:
        L = env.p.tax_levels
        x = b["gobs"][:T].reshape(T * E, env.G)[rows]
        valid = np.ones((len(rows), env.p.nb * L), bool)
        act = b["gact"].reshape(T * E, env.p.nb)[rows]
        lpo = b["glogp"].reshape(-1)[rows]
        vo = b["gvalue"][:T].reshape(-1)[rows]
        a, r = adv.reshape(-1)[rows], ret.reshape(-1)[rows]
        w = synth.unpack(wvec, env.G, H, env.p.nb * L)
        heads, head = env.p.nb, L
    return oppo.ppo_loss_grad64(w, x, act, valid, lpo, vo, a, r, clip=pp.clip, vf_coef=pp.vf_coef,
                                vclip=pp.vclip, ent_coef=pp.ent_coef, heads=heads, head=head)


@pytest.mark.parametrize("net", [0, 1])
def test_minibatch_gradient_matches_float64(net):
    """2 environments x 4 agents x 16 steps, 4 minibatches: the gradient of
    minibatch 1 of shuffle 3, every parameter tensor."""
    E, A, T = (2, 4, 16) if net == 0 else (8, 4, 16)
    env, pol, ro, ppo, b, pw, gw = _setup(E, A, T, seed=2, ppo_kw=dict(minibatches=4, seed=77),
                                          T_ep=12, T_tax=4)
    ppo.advantages(ro)
    grad, stats = ppo.minibatch_grad(ro, net, 3, 1)
    grad = grad.cpu().numpy()
    N = T * (E * A if net == 0 else E)
    rows = shuffle.minibatch_rows(1, 4, N, 77, 3)
    adv, ret, gadv, gret = _oracle_gae(env, b, ppo.pp)
    loss, g64, st = _oracle_grad(env, b, ppo.pp, net, rows, adv if net == 0 else gadv,
                                 ret if net == 0 else gret, pw if net == 0 else gw)
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
    gg = synth.unpack(grad, in_dim, H, O)
    for k, ref in g64.items():
        tol = 1e-3 * np.abs(ref).max() + 1e-7
        assert np.max(np.abs(gg[k].reshape(ref.shape) - ref)) <= tol, k
    # padding of the gradient vector is zero
    layout, n = synth.net_offsets(in_dim, H, O)
    used = np.zeros(n, bool)
    for _, shape, _, off in layout:
        used[off:off + int(np.prod(shape))] = True
    assert not grad[~used].any()
    s = stats.cpu().numpy()
    a_rows = (adv if net == 0 else gadv).reshape(-1)[rows]
    assert s[0] == pytest.approx(a_rows.sum(), abs=1e-4 * (1 + np.abs(a_rows).sum()))
    assert s[2] / len(rows) == pytest.approx(st["pg"], abs=1e-4 * (1 + abs(st["pg"])))
    assert s[4] / len(rows) == pytest.approx(st["ent"], rel=1e-4)


def test_update_is_one_adam_step_per_minibatch():
    """epochs = minibatches = 1: the update equals Adam's first step on the
    float64 gradient of the whole batch."""
    E, A, T = 2, 4, 12
    env, pol, ro, ppo, b, pw, gw = _setup(E, A, T, seed=5, ppo_kw=dict(minibatches=1, epochs=1, seed=3),
                                          T_ep=10, T_tax=5)
    before = [pol.pop_w.clone(), pol.gov_w.clone()]
    stats = ppo.update(ro).cpu().numpy()
    assert np.all(np.isfinite(stats))
    adv, ret, gadv, gret = _oracle_gae(env, b, ppo.pp)
    lr, eps = ppo.pp.lr, ppo.pp.eps
    for net, wvec, after in ((0, pw, pol.pop_w), (1, gw, pol.gov_w)):
        N = T * (E * A if net == 0 else E)
        rows = shuffle.minibatch_rows(0, 1, N, 3, 0 if net == 0 else 0x80000000)
        _, g64, st = _oracle_grad(env, b, ppo.pp, net, rows, adv if net == 0 else gadv,
                                  ret if net == 0 else gret, wvec)
        in_dim = env.D if net == 0 else env.G
        O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
        delta = synth.unpack(after.cpu().numpy() - before[net].cpu().numpy(), in_dim, H, O)
        w0 = synth.unpack(wvec, in_dim, H, O)
        for k, g in g64.items():
            # Adam's first step: -lr g / (|g| + eps); insensitive to gradient error where |g| >> eps
            expect = oppo.adam64(w0[k], g, np.zeros_like(g), np.zeros_like(g), 1, lr, eps=eps)[0] - w0[k]
            big = np.abs(g) > 1e-2 * np.abs(g).max() + 100 * eps
            d = delta[k].reshape(g.shape)
            assert np.allclose(d[big], expect[big], rtol=0, atol=2e-7), k
            assert np.all(np.abs(d) <= lr * 1.0001), k
        assert stats[net, 0] == pytest.approx(st["pg"], abs=1e-3 * (1 + abs(st["pg"])))


# Section 5's 4-resource market (prices 3, 6, 9, no taxes, skills growing
# around 1), and the largest market the PPO calls take (inputs and logits at
# most 128): 16 resources at 3 price levels, 123 inputs, 114 logits
MARKETS = {
    "r4": dict(R=4, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=2, gov_enabled=0, skill_gain=0.005,
               skill_init=1, T_ep=12, T_tax=4),
    "r16": dict(R=16, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=3, gov_enabled=0, skill_gain=0.005,
                skill_init=1, T_ep=12, T_tax=4),
}


@pytest.mark.parametrize("net,market,H2", [(0, "r4", 256), (1, "r4", 256), (0, "r16", 256),
                                           (0, "r4", 32), (1, "r4", 96), (0, "r16", 96)])
def test_fp32_gradient_widths_match_float64(net, market, H2):
    """Section 5's networks of 256 units, the smallest width (32) and one
    that is not a power of two (96): the float32 minibatch gradient against
    the float64 oracle, every parameter tensor, within 1e-3 of the tensor's
    largest entry, on minibatches of 60 to 80 rows (two or three 32-row
    tiles, the last one ragged; at 256 the weight-gradient kernel spans 2 x 2
    output tiles of 128)."""
    import paper_2410_22165_gb300 as P
    kw = MARKETS[market]
    E, A, T = (3, 5, 16) if net == 0 else (15, 4, 16)
    env = P.VecEnv(E, A, **kw)
    O_gov = env.p.nb * env.p.tax_levels
    pw = synth.net_weights(4, 0, env.D, H2, env.nA)
    gw = synth.net_weights(4, 1, env.G, H2, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H2)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=4)
    ro.run()
    ppo = P.PPO(pol, T, minibatches=4, seed=77)
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    ppo.advantages(ro)
    grad = ppo.minibatch_grad(ro, net, 3, 1)[0].cpu().numpy()
    N = T * (E * A if net == 0 else E)
    rows = shuffle.minibatch_rows(1, 4, N, 77, 3)
    adv, ret, gadv, gret = _oracle_gae(env, b, ppo.pp)
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else O_gov
    if net == 0:
        x = b["obs"][:T].reshape(T * E * A, env.D)[rows]
        valid = op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows]
        act, lpo = b["act"].reshape(-1, 1)[rows], b["logp"].reshape(-1)[rows]
        vo, a, r = b["value"][:T].reshape(-1)[rows], adv.reshape(-1)[rows], ret.reshape(-1)[rows]
        heads, head = 1, env.nA
    else:
        x = b["gobs"][:T].reshape(T * E, env.G)[rows]
        valid = np.ones((len(rows), O_gov), bool)
        act, lpo = b["gact"].reshape(T * E, env.p.nb)[rows], b["glogp"].reshape(-1)[rows]
        vo, a, r = b["gvalue"][:T].reshape(-1)[rows], gadv.reshape(-1)[rows], gret.reshape(-1)[rows]
        heads, head = env.p.nb, env.p.tax_levels
    w = synth.unpack(pw if net == 0 else gw, in_dim, H2, O)
    _, g64, _ = oppo.ppo_loss_grad64(w, x, act, valid, lpo, vo, a, r, clip=ppo.pp.clip, vf_coef=ppo.pp.vf_coef,
                                     vclip=ppo.pp.vclip, ent_coef=ppo.pp.ent_coef, heads=heads, head=head)
    gg = synth.unpack(grad, in_dim, H2, O)
    for k, ref in g64.items():
        tol = 1e-3 * np.abs(ref).max() + 1e-7
        assert np.max(np.abs(gg[k].reshape(ref.shape) - ref)) <= tol, k
    assert (env.D, env.nA) == ((39, 30) if market == "r4" else (123, 114))


def test_bf16_gradient_refuses_hidden_256():
    """The BF16 gradient takes hidden 128 only: hidden 256 is refused on the
    host before anything runs (EJ_ERR_UNSUPPORTED)."""
    import ctypes as C
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    env = P.VecEnv(2, 4, R=12, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=3, gov_enabled=0)
    pp = N.EjPpoParams()
    N.load().ej_ppo_params_default(C.byref(pp))
    fake = C.c_void_p(4096)
    b = N.EjRollout(**{f: 4096 for f, _ in N.EjRollout._fields_})
    st = N.load().ppo_minibatch_grad(C.byref(env.p), C.byref(pp), 8, 256, N.BF16, 0, fake, C.byref(b), fake,
                                     0, 0, fake, None, None)
    assert st == 3
