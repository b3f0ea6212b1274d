"""The hand-written actor-critic backward behind torch.autograd (PPOLoss).

Checks, on a 2-environment x 4-agent slice: autograd returns the library's
gradient; the loss equals the float64 oracle's loss of the same minibatch;
and the gradient agrees with central finite differences of the library's own
loss along the gradient direction and along a random direction.
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


def _setup(E=2, A=4, T=16, seed=2):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, T_ep=12, T_tax=4)
    O_gov = env.p.nb * env.p.tax_levels
    pw = synth.net_weights(seed, 0, env.D, H, env.nA)
    gw = synth.net_weights(seed, 1, env.G, H, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=seed)
    ro.run()
    ppo = P.PPO(pol, T, minibatches=4, seed=77)
    ppo.advantages(ro)
    return env, pol, ro, ppo, pw


def test_autograd_returns_library_gradient_and_oracle_loss():
    env, pol, ro, ppo, pw = _setup()
    w = pol.pop_w.clone().requires_grad_(True)
    loss = ppo.loss(w, ro, 0, 3, 1)
    (2.0 * loss).backward()
    grad, _ = ppo.minibatch_grad(ro, 0, 3, 1)
    assert torch.equal(w.grad, 2.0 * grad)
    # the same minibatch's loss in float64 on the CPU
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    E, A, T = env.E, env.A, ro.T
    done = np.repeat(b["done"][:, :, None], A, axis=2).reshape(T, E * A)
    adv, ret = oppo.gae64(b["rew"].reshape(T, E * A), b["value"].reshape(T + 1, E * A), done,
                          ppo.pp.gamma, ppo.pp.lam)
    rows = shuffle.minibatch_rows(1, 4, T * E * A, 77, 3)
    x = b["obs"][:T].reshape(T * E * A, env.D)[rows]
    valid = op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows]
    ref, _, _ = oppo.ppo_loss_grad64(synth.unpack(pw, env.D, H, env.nA), x, b["act"].reshape(-1, 1)[rows],
                                     valid, b["logp"].reshape(-1)[rows], b["value"][:T].reshape(-1)[rows],
                                     adv.reshape(-1)[rows], ret.reshape(-1)[rows], clip=ppo.pp.clip,
                                     vf_coef=ppo.pp.vf_coef, vclip=ppo.pp.vclip, ent_coef=ppo.pp.ent_coef,
                                     heads=1, head=env.nA)
    assert float(loss.detach()) == pytest.approx(ref, rel=1e-4, abs=1e-5)


@pytest.mark.parametrize("net", [0, 1])
def test_gradient_matches_finite_differences(net):
    env, pol, ro, ppo, _ = _setup(E=4 if net else 2)
    w0 = (pol.pop_w if net == 0 else pol.gov_w).clone()
    w = w0.clone().requires_grad_(True)
    ppo.loss(w, ro, net, 5, 2).backward()
    g = w.grad.double()
    gen = torch.Generator(device="cpu").manual_seed(11)
    rnd = torch.randn(w0.numel(), generator=gen, dtype=torch.float64).to(w0.device)
    rnd *= (g != 0).double()          # stay off the padding of the parameter vector
    for d in (g / g.norm(), rnd / rnd.norm()):
        slope = float(g @ d)
        L0 = float(ppo.loss(w0, ro, net, 5, 2))
        h = 1e-3 * max(abs(L0), 1e-2) / max(float(g.norm()), 1e-12)
        lp = float(ppo.loss((w0.double() + h * d).float(), ro, net, 5, 2))
        lm = float(ppo.loss((w0.double() - h * d).float(), ro, net, 5, 2))
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(slope, rel=2e-2, abs=2e-3 * float(g.norm())), (fd, slope)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_library_loss_entry(precision):
    """Entry 7 of the minibatch statistics is the loss of Section 4 assembled
    in the library: (policy loss + vf_coef value loss - ent_coef entropy) / n;
    the data-parallel form divides by the union's rows (moments[0])."""
    import paper_2410_22165_gb300 as P
    env, pol, ro, _, _ = _setup(E=4)
    ppo = P.PPO(pol, ro.T, precision=precision, minibatches=4, seed=77)
    ppo.advantages(ro)
    pp = ppo.pp
    for net in (0, 1):
        _, st = ppo.minibatch_grad(ro, net, 3, 1)
        n = ppo.minibatch_rows(net, 1)
        s = st.cpu().numpy()
        assert s[7] == pytest.approx((s[2] + pp.vf_coef * s[3] - pp.ent_coef * s[4]) / n, rel=1e-12)
        mom = ppo.minibatch_moments(ro, net, 3, 1)
        mom2 = mom.clone()
        mom2[0] *= 2                                   # as if a second rank held as many rows
        _, sg = ppo.minibatch_grad(ro, net, 3, 1, moments=mom2)
        g = sg.cpu().numpy()
        assert g[7] == pytest.approx((g[2] + pp.vf_coef * g[3] - pp.ent_coef * g[4]) / (2 * n), rel=1e-12)
