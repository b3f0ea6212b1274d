"""Parity of the policy forward, the sampler and the rollout with the oracle.

Float32 forward tolerance, derived from the arithmetic: every output is a
chain of three dot products of lengths K1 = in, K2 = K3 = H; with float32
rounding u = 2^-24 its error is at most (K1 + K2 + K3) u times the magnitude
obtained by running the network on |x| with |W| and |b| (float64).
BF16 forward tolerance: every product of a layer has both operands rounded to
bfloat16 (relative error <= 2^-9 each) and the activations between layers are
rounded again; over three layers the error is at most 8 * 2^-9 times the same
magnitude (accumulation is float32 and contributes far less).
Sampled actions are integers decided by float32 arithmetic: the oracle
takes the same decision in float32 (same exp, same summation order) from
the GPU's logits and must agree exactly.
"""
import numpy as np
import pytest

import synth
from oracle import policy as op
from oracle.env import default_params
from tests.parity import compare_env, oracle_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _mods():
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    return P, N


def magnitude(w, x):
    """Network outputs with every term replaced by its absolute value (float64)."""
    a = {k: np.abs(v) for k, v in w.items()}
    x = np.abs(np.asarray(x, np.float64))
    h = x @ a["W1"] + a["b1"]
    h = h @ a["W2"] + a["b2"]
    lg = h @ a["W3"] + a["b3"]
    g = x @ a["V1"] + a["c1"]
    g = g @ a["V2"] + a["c2"]
    v = (g @ a["V3"] + a["c3"])[:, 0]
    return lg, v


def _setup(E, A, seed=0, steps=37, precision="fp32", hidden=None, **kw):
    P, N = _mods()
    env = P.VecEnv(E, A, **kw)
    env.reset(seed=seed)
    out = env.step(steps)                       # in-kernel random play to reach varied states
    obs = out["obs"][-1].contiguous()
    gobs = out["gobs"][-1].contiguous()
    mask = out["mask"][-1].contiguous()
    D, G = env.D, env.G
    O_pop, O_gov = env.nA, env.p.nb * env.p.tax_levels
    hid = H if hidden is None else hidden
    pw = synth.net_weights(seed, 0, D, hid, O_pop)
    gw = synth.net_weights(seed, 1, G, hid, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=hid, precision=precision)
    return env, pol, obs, gobs, mask, pw, gw


def _bound(precision, in_dim):
    return (in_dim + 2 * H) * 2.0 ** -24 if precision == "fp32" else 8 * 2.0 ** -9


def _check_forward(logits, value, w, x, in_dim, precision="fp32"):
    lg64, v64 = op.mlp64(w, x)
    mlg, mv = magnitude(w, x)
    bound = _bound(precision, in_dim)
    assert np.all(np.abs(logits - lg64) <= bound * mlg + 1e-30), np.max(np.abs(logits - lg64) / mlg)
    assert np.all(np.abs(value - v64) <= bound * mv + 1e-30)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_population_forward_and_sampling(precision):
    E, A = 3, 37
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, precision=precision)
    P, N = _mods()
    out = pol.forward(N.NET_POP, obs, mask, logits=True, entropy=True)
    lg = out["logits"].cpu().numpy()
    val = out["value"].cpu().numpy()
    x = obs.cpu().numpy().reshape(E * A, env.D)
    w = synth.unpack(pw, env.D, H, env.nA)
    _check_forward(lg, val, w, x, env.D, precision)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    g = int(env.field("gstep")[0].item())
    u = synth.pop_draws(0, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)
    act = op.sample32(lg, valid, u)
    got = out["act"].cpu().numpy()[:, 0]
    assert np.array_equal(got, act)
    lp, ent = op.logp_entropy64(lg, valid, got)
    assert np.allclose(out["logp"].cpu().numpy(), lp, rtol=0, atol=1e-5 * (1 + np.abs(lp)).max())
    assert np.allclose(out["entropy"].cpu().numpy(), ent, rtol=0, atol=1e-5 * (1 + np.abs(ent)).max())


@pytest.mark.parametrize("levels", [5, 10, 20])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_population_forward_price_grids(precision, levels):
    """24, 44 and 84 actions (1, 2 and 3 mask words), 7 x 100 rows: several
    tiles and a ragged one."""
    P, N = _mods()
    E, A = 7, 100
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=5, precision=precision, T_ep=60, T_tax=10,
                                               **P.price_grid(levels))
    assert env.W == (env.nA + 31) // 32
    out = pol.forward(N.NET_POP, obs, mask, logits=True, entropy=True)
    lg = out["logits"].cpu().numpy()
    x = obs.cpu().numpy().reshape(E * A, env.D)
    _check_forward(lg, out["value"].cpu().numpy(), synth.unpack(pw, env.D, H, env.nA), x, env.D, precision)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    g = int(env.field("gstep")[0].item())
    u = synth.pop_draws(5, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)
    got = out["act"].cpu().numpy()[:, 0]
    assert np.array_equal(got, op.sample32(lg, valid, u))
    lp, ent = op.logp_entropy64(lg, valid, got)
    assert np.allclose(out["logp"].cpu().numpy(), lp, rtol=0, atol=1e-5 * (1 + np.abs(lp)).max())
    assert np.allclose(out["entropy"].cpu().numpy(), ent, rtol=0, atol=1e-5 * (1 + np.abs(ent)).max())


def test_segments_equal_separate_calls():
    """policy_forward_segments over several environments sets and both
    networks (one launch of up to 4 networks) equals one policy_forward per
    set, bit for bit."""
    import ctypes as C
    P, N = _mods()
    from paper_2410_22165_gb300.env import _ptr, _stream
    sets = []
    for k, (levels, E, A) in enumerate([(5, 3, 50), (10, 2, 37), (20, 4, 10), (5, 5, 20)]):
        env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=20 + k, precision="bf16", T_ep=30, T_tax=7,
                                                   **P.price_grid(levels))
        if k == 3:    # same population weights as set 0: one network
            pol = P.Policy(env, sets[0][1].pop_w.cpu(), sets[0][1].gov_w.cpu(), hidden=H, precision="bf16")
            pol.pop_w, pol.gov_w = sets[0][1].pop_w, sets[0][1].gov_w
        sets.append((env, pol, obs, gobs, mask))
    segs = []
    for env, pol, obs, gobs, mask in sets:
        for net in (N.NET_POP, N.NET_GOV):
            rows = env.E * env.A if net == N.NET_POP else env.E
            heads = 1 if net == N.NET_POP else env.p.nb
            segs.append(dict(env=env, net=net, w=pol.pop_w if net == N.NET_POP else pol.gov_w,
                             x=obs if net == N.NET_POP else gobs, mask=mask if net == N.NET_POP else None,
                             act=torch.empty((rows, heads), dtype=torch.int32, device="cuda"),
                             logp=torch.empty(rows, device="cuda"), value=torch.empty(rows, device="cuda"),
                             pol=pol))
    n = len(segs)
    V = C.c_void_p * n
    N.check(N.load().policy_forward_segments(
        n, V(*[C.addressof(s["env"].p) for s in segs]), V(*[_ptr(s["env"].state) for s in segs]),
        (C.c_int32 * n)(*[s["net"] for s in segs]), V(*[_ptr(s["w"]) for s in segs]), H, N.BF16,
        V(*[_ptr(s["x"]) for s in segs]), V(*[_ptr(s["mask"]) for s in segs]), V(*[_ptr(s["act"]) for s in segs]),
        V(*[_ptr(s["logp"]) for s in segs]), V(*[_ptr(s["value"]) for s in segs]), _stream()),
        "policy_forward_segments")
    for s in segs:
        ref = s["pol"].forward(s["net"], s["x"], s["mask"])
        assert torch.equal(ref["act"], s["act"]) and torch.equal(ref["logp"], s["logp"])
        assert torch.equal(ref["value"], s["value"])


@pytest.mark.parametrize("net", [0, 1])
def test_unaligned_observations(net):
    """Observation buffers 1, 2 and 3 floats past a 16-byte boundary (e.g.
    rollout slots of E x A x D floats) give the aligned buffer's results."""
    P, N = _mods()
    E, A = 5, 77
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=6, precision="bf16", T_ep=40, T_tax=9)
    x = obs if net == 0 else gobs
    ref = pol.forward(net, x, mask if net == 0 else None, logits=True, entropy=True)
    for off in (1, 2, 3):
        big = torch.zeros(x.numel() + 4, device="cuda")
        xs = big[off:off + x.numel()].view(x.shape)
        xs.copy_(x)
        assert xs.data_ptr() % 16 == 4 * off
        got = pol.forward(net, xs, mask if net == 0 else None, logits=True, entropy=True)
        for k in ref:
            assert torch.equal(ref[k], got[k]), (off, k)


def test_more_sets_than_one_launch_takes():
    """40 sets of two networks (20 small environments, shared weights): the
    call splits them into launches of at most 32 sets; results equal one
    policy_forward per set."""
    import ctypes as C
    P, N = _mods()
    from paper_2410_22165_gb300.env import _ptr, _stream
    rng = np.random.default_rng(3)
    base = None
    segs = []
    for k in range(20):
        E, A = int(rng.integers(1, 4)), int(rng.integers(5, 40))
        env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=40 + k, precision="bf16", T_ep=30, T_tax=7)
        if base is None:
            base = pol
        pol = P.Policy(env, base.pop_w.cpu(), base.gov_w.cpu(), hidden=H, precision="bf16")
        pol.pop_w, pol.gov_w = base.pop_w, base.gov_w
        for net in (N.NET_POP, N.NET_GOV):
            rows = E * A if net == N.NET_POP else E
            heads = 1 if net == N.NET_POP else env.p.nb
            segs.append(dict(env=env, pol=pol, net=net, x=obs if net == N.NET_POP else gobs,
                             mask=mask if net == N.NET_POP else None,
                             act=torch.empty((rows, heads), dtype=torch.int32, device="cuda"),
                             logp=torch.empty(rows, device="cuda"), value=torch.empty(rows, device="cuda")))
    n = len(segs)
    V = C.c_void_p * n
    N.check(N.load().policy_forward_segments(
        n, V(*[C.addressof(s["env"].p) for s in segs]), V(*[_ptr(s["env"].state) for s in segs]),
        (C.c_int32 * n)(*[s["net"] for s in segs]),
        V(*[_ptr(s["pol"].pop_w if s["net"] == N.NET_POP else s["pol"].gov_w) for s in segs]), H, N.BF16,
        V(*[_ptr(s["x"]) for s in segs]), V(*[_ptr(s["mask"]) for s in segs]), V(*[_ptr(s["act"]) for s in segs]),
        V(*[_ptr(s["logp"]) for s in segs]), V(*[_ptr(s["value"]) for s in segs]), _stream()),
        "policy_forward_segments")
    for s in segs:
        ref = s["pol"].forward(s["net"], s["x"], s["mask"])
        assert torch.equal(ref["act"], s["act"]) and torch.equal(ref["logp"], s["logp"])
        assert torch.equal(ref["value"], s["value"])


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_split_rollout_equals_one_chain(precision):
    """rollout_split: 2 and 3 chains of environments (ranges of 6 and 4/4/5
    of 13) on their own streams give the single chain's buffers and state bit
    for bit, eager and from a captured graph."""
    P, N = _mods()
    E, A, T = 13, 20, 6
    out = {}
    for chains in (1, 2, 3):
        env = P.VecEnv(E, A, T_ep=5, T_tax=3)
        pw = synth.net_weights(12, 0, env.D, H, env.nA)
        gw = synth.net_weights(12, 1, env.G, H, env.p.nb * env.p.tax_levels)
        pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H, precision=precision)
        ro = P.Rollout(env, pol, T)
        ro.chains = chains
        ro.reset(seed=12)
        ro.run()
        ro.capture()            # carry-over + one more rollout eagerly, then the graph
        ro.replay()
        torch.cuda.synchronize()
        out[chains] = ({k: v.clone() for k, v in ro.buf.items()}, env.state.clone())
    for chains in (2, 3):
        for k, v in out[1][0].items():
            assert torch.equal(v, out[chains][0][k]), (chains, k)
        assert torch.equal(out[1][1], out[chains][1])


@pytest.mark.parametrize("hidden,levels", [(64, 5), (64, 10), (128, 30), (256, 5), (256, 10)])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_forward_outside_the_pipelined_kernel(precision, hidden, levels):
    """Shapes the pipelined BF16 kernel does not take: hidden 64 (24 and 44
    actions), 124 actions at hidden 128 (P = 30 levels, 4 mask words) and
    hidden 256 (the two-CTA cluster kernel; 300 rows: three tiles, the last
    ragged); population and government networks against the oracle."""
    P, _ = _mods()
    _forward_vs_oracle(precision, hidden, P.price_grid(levels))


@pytest.mark.parametrize("R,Rd", [(4, 2), (12, 3)])
def test_section5_networks_of_256_units_fp32(R, Rd):
    """Section 5's networks of 256 units per layer on its multi-resource
    environments (30 and 86 actions), FP32 forward against the oracle."""
    _forward_vs_oracle("fp32", 256, dict(R=R, P=3, price_tick=3.0, price_ticks=[1, 2, 3], Rd=Rd,
                                         gov_enabled=0, skill_gain=0.005, skill_init=1))


@pytest.mark.parametrize("hidden", [32, 96])
def test_fp32_forward_small_and_odd_widths(hidden):
    """The smallest hidden width (32) and one that is not a power of two
    (96: three warp tiles across the columns), FP32 forward and sampling
    against the oracle."""
    _forward_vs_oracle("fp32", hidden, {})


def test_largest_market_fp32_hidden_256():
    """The largest market under 256 actions (16 resources at 7 price levels:
    123 inputs, 242 logits, 8 mask words) at hidden 256: the FP32 forward's
    largest tile of shared memory, against the oracle."""
    _forward_vs_oracle("fp32", 256, dict(R=16, P=7, price_tick=3.0, price_ticks=list(range(1, 8)), Rd=3,
                                         gov_enabled=0))


def test_section5_networks_of_256_units_bf16():
    """Section 5's 4-resource market (39 inputs, 46 actions) with networks of
    256 units in BF16 (the cluster kernel) against the oracle; the
    12-resource market's 95 inputs exceed the kernel's 64-column input operand
    and are refused before anything is launched."""
    s5 = dict(P=3, price_tick=3.0, price_ticks=[1, 2, 3], gov_enabled=0, skill_gain=0.005, skill_init=1)
    _forward_vs_oracle("bf16", 256, dict(R=4, Rd=2, **s5))
    P, N = _mods()
    env = P.VecEnv(2, 10, R=12, Rd=3, **s5)
    pw = torch.from_numpy(synth.net_weights(1, 0, env.D, 256, env.nA))
    gw = torch.from_numpy(synth.net_weights(1, 1, env.G, 256, env.p.nb * env.p.tax_levels))
    with pytest.raises(N.EjError, match="UNSUPPORTED"):
        P.Policy(env, pw, gw, hidden=256, precision="bf16").forward(N.NET_POP, torch.zeros((2, 10, env.D), device="cuda"))


def _forward_vs_oracle(precision, hidden, env_kw):
    P, N = _mods()
    E, A = 5, 60
    env = P.VecEnv(E, A, T_ep=40, T_tax=9, **env_kw)
    env.reset(seed=31)
    o = env.step(11)
    obs, gobs, mask = o["obs"][-1].contiguous(), o["gobs"][-1].contiguous(), o["mask"][-1].contiguous()
    O_gov = env.p.nb * env.p.tax_levels
    pw = synth.net_weights(31, 0, env.D, hidden, env.nA)
    gw = synth.net_weights(31, 1, env.G, hidden, O_gov)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=hidden, precision=precision)
    g = int(env.field("gstep")[0].item())
    bound = (env.D + 2 * hidden) * 2.0 ** -24 if precision == "fp32" else 8 * 2.0 ** -9
    # population
    out = pol.forward(N.NET_POP, obs, mask, logits=True)
    lg, val = out["logits"].cpu().numpy(), out["value"].cpu().numpy()
    x = obs.cpu().numpy().reshape(E * A, env.D)
    w = synth.unpack(pw, env.D, hidden, env.nA)
    lg64, v64 = op.mlp64(w, x)
    mlg, mv = magnitude(w, x)
    assert np.all(np.abs(lg - lg64) <= bound * mlg + 1e-30) and np.all(np.abs(val - v64) <= bound * mv + 1e-30)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    u = synth.pop_draws(31, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)
    assert np.array_equal(out["act"].cpu().numpy()[:, 0], op.sample32(lg, valid, u))
    # government
    out = pol.forward(N.NET_GOV, gobs, logits=True)
    lg = out["logits"].cpu().numpy()
    wg = synth.unpack(gw, env.G, hidden, O_gov)
    lg64, v64 = op.mlp64(wg, gobs.cpu().numpy())
    mlg, mv = magnitude(wg, gobs.cpu().numpy())
    assert np.all(np.abs(lg - lg64) <= bound * mlg + 1e-30)
    _, gu = synth.gov_draws(31, np.arange(E), g, 1, env.p.nb, env.p.tax_levels)
    L = env.p.tax_levels
    for b in range(env.p.nb):
        head = lg[:, b * L:(b + 1) * L]
        assert np.array_equal(out["act"].cpu().numpy()[:, b], op.sample32(head, np.ones_like(head, bool), gu[0, :, b]))


def test_bf16_shape_limits_are_reported():
    """BF16 at hidden 64 takes at most 63 logits: 84 actions are refused with
    EJ_ERR_UNSUPPORTED (nothing launched); FP32 takes the shape."""
    P, N = _mods()
    env = P.VecEnv(2, 10, **P.price_grid(20))
    env.reset(seed=1)
    pw = torch.from_numpy(synth.net_weights(1, 0, env.D, 64, env.nA))
    gw = torch.from_numpy(synth.net_weights(1, 1, env.G, 64, env.p.nb * env.p.tax_levels))
    obs = torch.zeros((2, 10, env.D), device="cuda")
    with pytest.raises(N.EjError, match="UNSUPPORTED"):
        P.Policy(env, pw, gw, hidden=64, precision="bf16").forward(N.NET_POP, obs)
    out = P.Policy(env, pw, gw, hidden=64, precision="fp32").forward(N.NET_POP, obs)
    assert torch.isfinite(out["value"]).all()


def test_given_uniforms_and_values_only():
    E, A = 2, 64
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=4)
    P, N = _mods()
    u = torch.rand(E * A, 1, device="cuda")
    out = pol.forward(N.NET_POP, obs, mask, u=u, logits=True)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)
    act = op.sample32(out["logits"].cpu().numpy(), valid, u.cpu().numpy()[:, 0])
    assert np.array_equal(out["act"].cpu().numpy()[:, 0], act)
    v_only = pol.forward(N.NET_POP, obs, mask, sample=False)
    assert torch.equal(v_only["value"], out["value"])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_government_forward_and_sampling(precision):
    E, A = 170, 10                    # 170 government rows: full tiles and a ragged one
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=2, precision=precision, T_ep=50, T_tax=10)
    P, N = _mods()
    out = pol.forward(N.NET_GOV, gobs, logits=True, entropy=True)
    lg = out["logits"].cpu().numpy()
    L = env.p.tax_levels
    w = synth.unpack(gw, env.G, H, env.p.nb * L)
    _check_forward(lg, out["value"].cpu().numpy(), w, gobs.cpu().numpy(), env.G, precision)
    g = int(env.field("gstep")[0].item())
    _, gu = synth.gov_draws(2, np.arange(E), g, 1, env.p.nb, L)
    got = out["act"].cpu().numpy()
    lp_tot = np.zeros(E)
    for b in range(env.p.nb):
        head = lg[:, b * L:(b + 1) * L]
        valid = np.ones_like(head, bool)
        a = op.sample32(head, valid, gu[0, :, b])
        assert np.array_equal(got[:, b], a)
        lp, _ = op.logp_entropy64(head, valid, a)
        lp_tot += lp
    assert np.allclose(out["logp"].cpu().numpy(), lp_tot, atol=1e-5 * (1 + np.abs(lp_tot)).max())


@pytest.mark.parametrize("precision,hidden", [("fp32", 128), ("bf16", 128), ("bf16", 256)])
def test_rollout_matches_oracle_step_by_step(precision, hidden):
    """T = 25 steps across an episode end: every sampled action is the oracle's
    decision on the GPU's logits; the environment transitions equal the oracle
    run with the GPU's actions; stored values and log-probabilities are the
    policy's.  Hidden 256 in BF16 is the two-CTA cluster kernel."""
    E, A, T = 3, 20, 25
    kw = dict(T_ep=20, T_tax=5)
    P, N = _mods()
    env = P.VecEnv(E, A, **kw)
    pw = synth.net_weights(9, 0, env.D, hidden, env.nA)
    gw = synth.net_weights(9, 1, env.G, hidden, env.p.nb * env.p.tax_levels)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=hidden, precision=precision)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=9)
    b = {k: v.cpu().numpy() for k, v in ro.run().items()}
    torch.cuda.synchronize()
    # a second environment replays the observations through policy_forward
    probe = P.VecEnv(E, A, **kw)
    probe.reset(seed=9)
    pprobe = P.Policy(probe, torch.from_numpy(pw), torch.from_numpy(gw), hidden=hidden, precision=precision)
    wp = synth.unpack(pw, env.D, hidden, env.nA)
    L = env.p.tax_levels
    for t in range(T + 1):
        obs = torch.from_numpy(b["obs"][t]).cuda()
        mask = torch.from_numpy(b["mask"][t]).cuda()
        u = torch.from_numpy(synth.pop_draws(9, np.arange(E), A, t, 1, env.nA)[3][0].reshape(E * A, 1)).cuda()
        o = pprobe.forward(N.NET_POP, obs, mask, u=u, logits=True)
        assert np.array_equal(o["value"].cpu().numpy(), b["value"][t].reshape(-1))
        if t == T:
            break
        lg = o["logits"].cpu().numpy()
        valid = op.mask_bits(b["mask"][t].view(np.uint32).reshape(E * A, env.W), env.nA)
        assert np.array_equal(b["act"][t].reshape(-1), op.sample32(lg, valid, u.cpu().numpy()[:, 0]))
        assert np.array_equal(o["act"].cpu().numpy()[:, 0], b["act"][t].reshape(-1))
        assert np.array_equal(o["logp"].cpu().numpy(), b["logp"][t].reshape(-1))
        _check_forward(lg, o["value"].cpu().numpy(), wp, b["obs"][t].reshape(E * A, env.D), env.D, precision)
        _, gu = synth.gov_draws(9, np.arange(E), t, 1, env.p.nb, L)
        og = pprobe.forward(N.NET_GOV, torch.from_numpy(b["gobs"][t]).cuda(),
                            u=torch.from_numpy(gu[0]).cuda(), logits=True)
        assert np.array_equal(og["act"].cpu().numpy(), b["gact"][t])
    # environment transitions: the oracle stepped with the GPU's actions
    p = default_params(**kw)
    from oracle.env import OracleEnv
    for e in range(E):
        o = OracleEnv(p, A)
        inp = synth.episode_inputs(9, [e], A, p["R"], p["nb"], o.nA, p["tax_levels"], T, p["T_ep"])
        o.reset(inp["sg0"][0], inp["sc0"][0])
        ref = o.run(b["act"][:, e], b["gact"][:, e], inp["gather_u"][:, 0], inp["tb"][:, 0],
                    inp["later_sg"][:, 0], inp["later_sc"][:, 0])
        g = dict(rew=b["rew"][:, e], grew=b["grew"][:, e], done=b["done"][:, e],
                 obs=b["obs"][1:, e], gobs=b["gobs"][1:, e], mask=b["mask"][1:, e])
        compare_env(g, ref, env.params, A)


def test_no_device_fault_recorded():
    P, N = _mods()
    import ctypes as C
    f = C.c_int32(-1)
    N.check(N.load().ej_device_status(C.byref(f), 0), "ej_device_status")
    assert f.value == 0


def test_rollout_graph_replay_equals_eager():
    """A rollout captured as a CUDA graph and replayed gives the eager rollout's buffers."""
    import paper_2410_22165_gb300 as P
    E, A, T = 4, 10, 12
    res = []
    for graph in (False, True):
        env = P.VecEnv(E, A, T_ep=8, T_tax=4)
        pw = synth.net_weights(3, 0, env.D, 128, env.nA)
        gw = synth.net_weights(3, 1, env.G, 128, env.p.nb * env.p.tax_levels)
        pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=128, precision="bf16")
        ro = P.Rollout(env, pol, T)
        ro.reset(seed=5)
        ro.run()
        if graph:
            ro.capture()          # second rollout, eager
            ro.replay()           # third rollout, from the graph
        else:
            for _ in range(2):
                ro.carry_over()
                ro.run()
        torch.cuda.synchronize()
        res.append({k: v.clone() for k, v in ro.buf.items()})
    for k in res[0]:
        assert torch.equal(res[0][k], res[1][k]), k


@pytest.mark.parametrize("precision,hidden", [("fp32", 128), ("bf16", 128), ("bf16", 256)])
def test_full_size_forward_sampled_rows(precision, hidden):
    """The rollout workload's size, E = 4096 x A = 100 (409,600 rows, 3,200 tiles: every CTA and both
    warpgroup pipelines run many tiles; at hidden 256 every cluster): 3,000 sampled rows checked
    against the float64 forward, and every sampled action against the oracle's float32 sampler on the
    kernel's logits."""
    E, A = 4096, 100
    env, pol, obs, gobs, mask, pw, gw = _setup(E, A, seed=8, steps=5, precision=precision, hidden=hidden,
                                               T_ep=1000, T_tax=100)
    P, N = _mods()
    out = pol.forward(N.NET_POP, obs, mask, logits=True, entropy=True)
    rng = np.random.default_rng(8)
    rows = np.sort(rng.choice(E * A, 3000, replace=False))
    rows = np.concatenate([rows, [0, 127, 128, E * A - 1]])
    lg = out["logits"].cpu().numpy()[rows]
    val = out["value"].cpu().numpy()[rows]
    x = obs.cpu().numpy().reshape(E * A, env.D)[rows]
    _check_forward(lg, val, synth.unpack(pw, env.D, hidden, env.nA), x, env.D, precision)
    valid = op.mask_bits(mask.cpu().numpy().view(np.uint32).reshape(E * A, env.W), env.nA)[rows]
    g = int(env.field("gstep")[0].item())
    u = synth.pop_draws(8, np.arange(E), A, g, 1, env.nA)[3][0].reshape(E * A)[rows]   # key = the reset seed
    assert np.array_equal(out["act"].cpu().numpy()[rows, 0], op.sample32(lg, valid, u))
