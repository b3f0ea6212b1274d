"""BF16 tensor-core PPO minibatch gradient against the float64 oracle.

The BF16 path rounds every GEMM operand (inputs, activations, weights,
backward signals) to bfloat16 (8-bit significand, unit roundoff 2^-9) and
accumulates in float32.  Two references:

* the oracle's BF16-operand form (ppo_loss_grad64 with operand=bf16_round:
  the same operands rounded, float64 products and sums).  What remains is
  float32 accumulation (K <= 128 per product, sums over tiles) and the rare
  operand that rounds to the neighbouring bfloat16 value because its float32
  and float64 values straddle a rounding boundary: per parameter tensor,
  relative L2 error <= 2e-3 and every entry within 1e-2 of the tensor's
  largest entry.
* the exact float64 gradient: here the rounding itself counts, including
  ReLU units whose pre-activation sign flips under rounding, which moves a
  whole term, so the error depends on the rows (a 32-row government slice
  reaches 0.1 relative L2 in W2).  The bound is derived per tensor: the
  kernel's distance from the exact gradient is at most the BF16-operand
  form's own distance from it plus the first reference's tolerance
  (measured values are printed).
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
TIGHT = (2e-3, 1e-2)        # against the BF16-operand oracle


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _setup(E, A, T, seed, ppo_kw, **kw):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, **kw)
    O_gov = env.p.nb * env.p.tax_levels
    pw = synth.net_weights(seed, 0, env.D, H, env.nA)
    gw = synth.net_weights(seed, 1, env.G, H, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=seed)
    ro.run()
    ppo = P.PPO(pol, T, precision="bf16", **ppo_kw)
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    return env, pol, ro, ppo, b, pw, gw


def _oracle(env, b, pp, net, rows, wvec, operand=None):
    E, A = env.E, env.A
    T = b["rew"].shape[0]
    if net == 0:
        done = np.repeat(b["done"][:, :, None], A, axis=2).reshape(T, E * A)
        adv, ret = oppo.gae64(b["rew"].reshape(T, E * A), b["value"].reshape(T + 1, E * A), done, pp.gamma, pp.lam)
        x = b["obs"][:T].reshape(T * E * A, env.D)[rows]
        valid = op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows]
        act = b["act"].reshape(-1, 1)[rows]
        lpo, vo = b["logp"].reshape(-1)[rows], b["value"][:T].reshape(-1)[rows]
        w = synth.unpack(wvec, env.D, H, env.nA)
        heads, head = 1, env.nA
    else:
        adv, ret = oppo.gae64(b["grew"], b["gvalue"], b["done"], pp.gamma, pp.lam)
        L = env.p.tax_levels
        x = b["gobs"][:T].reshape(T * E, env.G)[rows]
        valid = np.ones((len(rows), env.p.nb * L), bool)
        act = b["gact"].reshape(T * E, env.p.nb)[rows]
        lpo, vo = b["glogp"].reshape(-1)[rows], b["gvalue"][:T].reshape(-1)[rows]
        w = synth.unpack(wvec, env.G, H, env.p.nb * L)
        heads, head = env.p.nb, L
    return oppo.ppo_loss_grad64(w, x, act, valid, lpo, vo, adv.reshape(-1)[rows], ret.reshape(-1)[rows],
                                clip=pp.clip, vf_coef=pp.vf_coef, vclip=pp.vclip, ent_coef=pp.ent_coef,
                                heads=heads, head=head, operand=operand)


def _compare(env, net, grad, g64, tol, label):
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
    gg = synth.unpack(grad, in_dim, H, O)
    worst = {}
    for k, ref in g64.items():
        got = gg[k].reshape(ref.shape)
        l2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        mx = np.max(np.abs(got - ref)) / max(np.abs(ref).max(), 1e-30)
        worst[k] = (l2, mx)
        assert l2 <= tol[0] and mx <= tol[1], (label, k, l2, mx)
    layout, n = synth.net_offsets(in_dim, H, O)
    used = np.zeros(n, bool)
    for _, shape, _, off in layout:
        used[off:off + int(np.prod(shape))] = True
    assert not grad[~used].any()
    print(f"bf16 gradient vs {label} (rel L2, rel max):",
          {k: (float(f"{a:.2e}"), float(f"{b:.2e}")) for k, (a, b) in worst.items()})
    return worst


def _compare_exact(env, net, grad, gbf, g64):
    """The kernel against the exact gradient, per tensor: relative L2 and
    relative max error at most those of the BF16-operand form (gbf) plus
    TIGHT."""
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
    gg = synth.unpack(grad, in_dim, H, O)
    errs = {}
    for k, ref in g64.items():
        scale_l2, scale_mx = max(np.linalg.norm(ref), 1e-30), max(np.abs(ref).max(), 1e-30)
        got = gg[k].reshape(ref.shape)
        l2, mx = np.linalg.norm(got - ref) / scale_l2, np.max(np.abs(got - ref)) / scale_mx
        f_l2, f_mx = np.linalg.norm(gbf[k] - ref) / scale_l2, np.max(np.abs(gbf[k] - ref)) / scale_mx
        errs[k] = (float(f"{l2:.2e}"), float(f"{f_l2:.2e}"))
        assert l2 <= f_l2 + TIGHT[0] and mx <= f_mx + TIGHT[1], (k, l2, f_l2, mx, f_mx)
    print("bf16 gradient vs float64 oracle (kernel rel L2, BF16-operand form rel L2):", errs)


@pytest.mark.parametrize("net", [0, 1])
def test_bf16_gradient_small_slice(net):
    """One partial tile: 2 (or 8) environments x 4 agents x 16 steps, minibatch 1 of 4."""
    E, A, T = (2, 4, 16) if net == 0 else (8, 4, 16)
    env, pol, ro, ppo, b, pw, gw = _setup(E, A, T, 2, dict(minibatches=4, seed=77), T_ep=12, T_tax=4)
    ppo.advantages(ro)
    grad, stats = ppo.minibatch_grad(ro, net, 3, 1)
    N = T * (E * A if net == 0 else E)
    rows = shuffle.minibatch_rows(1, 4, N, 77, 3)
    wv = pw if net == 0 else gw
    loss, g64, st = _oracle(env, b, ppo.pp, net, rows, wv)
    _, gbf, _ = _oracle(env, b, ppo.pp, net, rows, wv, operand=oppo.bf16_round)
    _compare(env, net, grad.cpu().numpy(), gbf, TIGHT, "bf16-operand oracle")
    _compare_exact(env, net, grad.cpu().numpy(), gbf, g64)
    s = stats.cpu().numpy()
    assert s[2] / len(rows) == pytest.approx(st["pg"], abs=2e-2 * (1 + abs(st["pg"])))
    assert s[4] / len(rows) == pytest.approx(st["ent"], rel=2e-2)


@pytest.mark.parametrize("net", [0, 1])
def test_bf16_gradient_many_tiles_ragged(net):
    """Many 128-row tiles per CTA (accumulation across tiles in tensor memory)
    and a ragged last tile: 32 environments x 50 agents x 40 steps, minibatch 2
    of 3 (21,333 population rows); the government network sees 427 rows."""
    E, A, T = 32, 50, 40
    env, pol, ro, ppo, b, pw, gw = _setup(E, A, T, 4, dict(minibatches=3, seed=5), T_ep=30, T_tax=6)
    ppo.advantages(ro)
    grad, stats = ppo.minibatch_grad(ro, net, 9, 2)
    N = T * (E * A if net == 0 else E)
    rows = shuffle.minibatch_rows(2, 3, N, 5, 9)
    assert len(rows) % 128 != 0
    wv = pw if net == 0 else gw
    _, g64, _ = _oracle(env, b, ppo.pp, net, rows, wv)
    _, gbf, _ = _oracle(env, b, ppo.pp, net, rows, wv, operand=oppo.bf16_round)
    _compare(env, net, grad.cpu().numpy(), gbf, TIGHT, "bf16-operand oracle")
    _compare_exact(env, net, grad.cpu().numpy(), gbf, g64)


def test_bf16_update_moves_weights_like_fp32():
    """A whole BF16 update: finite statistics, and over 90 % of the parameter
    steps whose float32 step is not tiny have the float32 step's sign."""
    import paper_2410_22165_gb300 as P
    E, A, T = 4, 10, 32
    steps = {}
    for prec in ("fp32", "bf16"):
        env, pol, ro, _, b, pw, gw = _setup(E, A, T, 6, dict(minibatches=2, seed=1), T_ep=20, T_tax=5)
        ppo = P.PPO(pol, T, precision=prec, minibatches=2, epochs=1, seed=1)
        before = pol.pop_w.clone()
        stats = ppo.update(ro).cpu().numpy()
        assert np.all(np.isfinite(stats))
        steps[prec] = (pol.pop_w - before).cpu().numpy()
    big = np.abs(steps["fp32"]) > 0.5 * ppo.pp.lr
    agree = np.mean(np.sign(steps["fp32"][big]) == np.sign(steps["bf16"][big]))
    print("sign agreement of bf16 and fp32 update steps:", agree)
    assert agree > 0.9, agree


def test_bf16_gradient_profile_size_minibatch():
    """The PPO profile case's minibatch: E = 256 x A = 100 x 32 steps, minibatch 3 of 8 (102,400
    population rows = 800 tiles, several per CTA and role), against the BF16-operand oracle."""
    E, A, T = 256, 100, 32
    env, pol, ro, ppo, b, pw, gw = _setup(E, A, T, 7, dict(minibatches=8, seed=11), T_ep=1000, T_tax=100)
    ppo.advantages(ro)
    grad, _ = ppo.minibatch_grad(ro, 0, 2, 3)
    rows = shuffle.minibatch_rows(3, 8, T * E * A, 11, 2)
    _, gbf, _ = _oracle(env, b, ppo.pp, 0, rows, pw, operand=oppo.bf16_round)
    _compare(env, 0, grad.cpu().numpy(), gbf, TIGHT, "bf16-operand oracle")
