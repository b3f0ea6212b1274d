"""Pins of the GAE / PPO / Adam oracle (no GPU)."""
import numpy as np
import pytest

from oracle import ppo


def test_gae_constant_rewards_closed_form():
    """Constant r and V, no episode end: delta = r + (gamma - 1) V and
    A_t = delta (1 - (gamma lambda)^(T - t)) / (1 - gamma lambda)."""
    T, N, r, V, g, lam = 50, 3, 0.7, 2.0, 0.99, 0.95
    adv, ret = ppo.gae64(np.full((T, N), r), np.full((T + 1, N), V), np.zeros((T, N)), g, lam)
    delta = r + (g - 1) * V
    k = T - np.arange(T)
    expect = delta * (1 - (g * lam) ** k) / (1 - g * lam)
    assert np.allclose(adv[:, 0], expect, rtol=1e-12)
    assert np.allclose(ret, adv + V)


def test_gae_limits_and_episode_end():
    rng = np.random.default_rng(1)
    T, N, g = 20, 4, 0.9
    rew = rng.normal(size=(T, N)); val = rng.normal(size=(T + 1, N))
    done = np.zeros((T, N)); done[7, 1] = 1
    # lambda = 0: one-step TD error
    adv0, _ = ppo.gae64(rew, val, done, g, 0.0)
    nd = 1 - done
    assert np.allclose(adv0, rew + g * nd * val[1:] - val[:-1])
    # lambda = 1: discounted return (bootstrapped at T, cut at the episode end) minus V
    adv1, ret1 = ppo.gae64(rew, val, done, g, 1.0)
    G = val[T].copy()
    for t in range(T - 1, -1, -1):
        G = rew[t] + g * nd[t] * G
        assert np.allclose(ret1[t], G)


def _rand_problem(seed, heads=1, head=6, in_dim=5, H=8, N=16):
    rng = np.random.default_rng(seed)
    O = heads * head
    w = dict(W1=rng.normal(size=(in_dim, H)) * 0.5, b1=rng.normal(size=H) * 0.1,
             W2=rng.normal(size=(H, H)) * 0.4, b2=rng.normal(size=H) * 0.1,
             W3=rng.normal(size=(H, O)) * 0.4, b3=rng.normal(size=O) * 0.1,
             V1=rng.normal(size=(in_dim, H)) * 0.5, c1=rng.normal(size=H) * 0.1,
             V2=rng.normal(size=(H, H)) * 0.4, c2=rng.normal(size=H) * 0.1,
             V3=rng.normal(size=(H, 1)) * 0.4, c3=rng.normal(size=1) * 0.1)
    x = rng.normal(size=(N, in_dim))
    valid = rng.random((N, O)) < 0.7
    act = np.zeros((N, heads), int)
    for h in range(heads):
        valid[:, h * head] = True
        for i in range(N):
            act[i, h] = rng.choice(np.nonzero(valid[i, h * head:(h + 1) * head])[0])
    logp_old = rng.normal(size=N) * 0.3 - 1.5
    v_old = rng.normal(size=N)
    adv = rng.normal(size=N)
    ret = rng.normal(size=N) * 2
    return w, x, act, valid, logp_old, v_old, adv, ret


@pytest.mark.parametrize("heads,coef", [(1, dict(clip=0.2, vf_coef=0.25, vclip=10.0, ent_coef=0.1)),
                                        (1, dict(clip=0.05, vf_coef=1.0, vclip=0.1, ent_coef=0.0)),
                                        (3, dict(clip=0.2, vf_coef=0.25, vclip=10.0, ent_coef=0.1))])
def test_ppo_gradient_matches_finite_differences(heads, coef):
    """Hand-written backpropagation against central differences of the loss
    (float64), for every parameter tensor, including clipped ratios and a
    clipped value loss."""
    w, x, act, valid, lo, vo, adv, ret = _rand_problem(3 + heads, heads=heads)
    head = valid.shape[1] // heads
    f = lambda ww: ppo.ppo_loss_grad64(ww, x, act, valid, lo, vo, adv, ret, heads=heads, head=head, **coef)
    loss, g, st = f(w)
    rng = np.random.default_rng(9)
    h = 1e-6
    for k in w:
        flat = w[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            wp = {kk: vv.copy() for kk, vv in w.items()}
            wm = {kk: vv.copy() for kk, vv in w.items()}
            wp[k].reshape(-1)[idx] += h
            wm[k].reshape(-1)[idx] -= h
            fd = (f(wp)[0] - f(wm)[0]) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 3.0]); gr = np.array([0.5, -4.0, 1e-3])
    q, m, v = ppo.adam64(p, gr, np.zeros(3), np.zeros(3), 1, lr=1e-2, eps=1e-12)
    assert np.allclose(q, p - 1e-2 * np.sign(gr))


def test_bf16_round_matches_torch_bfloat16():
    """The oracle's bfloat16 rounding against torch's float32 -> bfloat16
    conversion (round to nearest, ties to even), including exact ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-30, 30, 4000),
                           [0.0, 1.0, -1.0, 0.5, 3.0, 1e-38, -2.5e38]])
    # float32 values exactly halfway between two bfloat16 values: low 16 bits 0x8000
    expo = rng.integers(100, 150, 500, dtype=np.uint64) << np.uint64(23)
    mant = rng.integers(0, 1 << 7, 500, dtype=np.uint64) << np.uint64(16)
    ties = (expo | mant | np.uint64(0x8000)).astype(np.uint32).view(np.float32).astype(np.float64)
    for v in (vals, ties, -ties):
        ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(ppo.bf16_round(v), ref)
    r = ppo.bf16_round(vals)
    assert np.array_equal(ppo.bf16_round(r), r)


def test_bf16_operand_form_reduces_to_exact_and_stays_close():
    """With the identity as operand rounding the BF16-operand form is the exact
    gradient; with bfloat16 rounding it differs from it, by a few per cent of
    the gradient's norm at most."""
    coef = dict(clip=0.2, vf_coef=0.25, vclip=10.0, ent_coef=0.1)
    w, x, act, valid, lo, vo, adv, ret = _rand_problem(5, heads=1)
    head = valid.shape[1]
    f = lambda **kw: ppo.ppo_loss_grad64(w, x, act, valid, lo, vo, adv, ret, heads=1, head=head, **coef, **kw)
    l0, g0, _ = f()
    l1, g1, _ = f(operand=lambda t: t)
    assert l0 == l1 and all(np.array_equal(g0[k], g1[k]) for k in g0)
    l2, g2, _ = f(operand=ppo.bf16_round)
    assert l2 == pytest.approx(l0, rel=5e-2)
    a = np.concatenate([g0[k].ravel() for k in g0])
    b = np.concatenate([g2[k].ravel() for k in g0])
    assert 0 < np.linalg.norm(b - a) <= 5e-2 * np.linalg.norm(a)


def test_union_moments_split_sums_to_whole_minibatch():
    """A minibatch split into two parts, each part given the moments of the
    whole: the parts' losses and gradients sum to the whole's (the loss is a
    mean over rows, so it is additive once the normalisation is shared); with
    the whole's own moments the whole is unchanged."""
    coef = dict(clip=0.2, vf_coef=0.25, vclip=10.0, ent_coef=0.1)
    w, x, act, valid, lo, vo, adv, ret = _rand_problem(7, heads=1, N=24)
    head = valid.shape[1]
    mom = (len(adv), adv.sum(), (adv * adv).sum())

    def f(sl, **kw):
        return ppo.ppo_loss_grad64(w, x[sl], act[sl], valid[sl], lo[sl], vo[sl], adv[sl], ret[sl], heads=1,
                                   head=head, **coef, **kw)
    l_all, g_all, _ = f(slice(None))
    l_same, g_same, _ = f(slice(None), moments=mom)
    assert l_same == pytest.approx(l_all, rel=1e-12)
    l_a, g_a, _ = f(slice(0, 9), moments=mom)
    l_b, g_b, _ = f(slice(9, None), moments=mom)
    assert l_a + l_b == pytest.approx(l_all, rel=1e-12)
    for k in g_all:
        assert np.allclose(g_a[k] + g_b[k], g_all[k], rtol=1e-10, atol=1e-14), k
        assert np.allclose(g_same[k], g_all[k], rtol=1e-12, atol=1e-15), k
