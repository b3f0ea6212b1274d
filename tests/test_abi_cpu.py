"""The C ABI library loads without a GPU, exports every symbol the header
declares, and validates parameters on the host."""
import ctypes as C
import os
import re

import pytest

from oracle.env import default_params
from paper_2410_22165_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2410_22165_gb300 import build
    build.build()
    return N.load()


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;]*\)\s*;", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("_")))


def test_header_symbols_exported(lib):
    names = declared_functions()
    assert {"env_reset", "env_step", "ej_sizes", "ej_params_default"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(N.exported_symbols()) <= set(names)


def test_defaults_match_table2_transcriptions(lib):
    """The library's defaults and the oracle's are two independent
    transcriptions of Table 2; they must agree."""
    p = N.params_dict(N.make_params())
    o = default_params()
    for k, v in o.items():
        if isinstance(v, float):
            assert p[k] == pytest.approx(v, rel=1e-7), k
        else:
            assert p[k] == v, k


def test_sizes(lib):
    s = N.sizes(N.make_params(E=1024, A=100))
    assert (s.n_actions, s.obs_dim, s.gobs_dim, s.mask_words) == (24, 25, 14, 1)
    assert s.threads == 128 and s.book_cap == 1500
    assert s.smem_bytes * 7 <= 227 * 1024 - 7 * 1024          # 7 CTAs per SM
    s = N.sizes(N.make_params(R=12, P=3, price_ticks=[1, 2, 3]))
    assert s.n_actions == 86


@pytest.mark.parametrize("bad", [dict(A=0), dict(A=2000), dict(R=0), dict(P=33), dict(nb=5),
                                 dict(T_ep=70000), dict(max_orders=17), dict(Rd=3),
                                 dict(price_ticks=[1, 1, 2, 3, 4]), dict(tax_levels=1),
                                 dict(eta=1.0), dict(price_tick=0.0)])
def test_invalid_params_rejected(lib, bad):
    p = N.make_params(**bad)
    s = N.EjSizes()
    st = lib.ej_sizes(C.byref(p), C.byref(s))
    assert st in (1, 3)
    assert lib.ej_last_error().decode()


def test_step_argument_checks(lib):
    p = N.make_params(E=2, A=10)
    # NULL state, and act without tb: rejected on the host before any launch
    assert lib.env_step(C.byref(p), None, 1, None, None, None, None, None, None, None, None,
                        None, None, None) == 1
    fake = C.c_void_p(256)
    # gather draws without tie-break keys, and draws without actions: rejected
    assert lib.env_step(C.byref(p), fake, 1, fake, None, fake, None, None, None, None, None,
                        None, None, None) == 1
    assert lib.env_step(C.byref(p), fake, 1, None, None, fake, fake, None, None, None, None,
                        None, None, None) == 1
    assert lib.env_step(C.byref(p), fake, -1, None, None, None, None, None, None, None, None,
                        None, None, None) == 1
    assert lib.env_step(C.byref(p), C.c_void_p(300), 1, None, None, None, None, None, None, None,
                        None, None, None, None) == 1                   # misaligned state
    assert lib.env_step(C.byref(p), fake, 0, None, None, None, None, None, None, None, None,
                        None, None, None) == 0                         # nothing to do


def test_state_layout(lib):
    p = N.make_params(E=3, A=10)
    s = N.sizes(p)
    prev_end = 0
    for f in N.FIELDS:
        off, cnt, esz = N.state_field(p, f)
        assert off % 256 == 0 and off >= prev_end and esz == 4
        prev_end = off + cnt * esz
    assert prev_end <= s.state_bytes


def test_net_layout_matches_generator(lib):
    import synth
    p = N.make_params(E=4, A=10)
    s = N.sizes(p)
    for net, (i, o) in ((N.NET_POP, (s.obs_dim, s.n_actions)), (N.NET_GOV, (s.gobs_dim, 3 * 21))):
        for H in (32, 128, 256):
            n = C.c_uint64()
            assert lib.ej_net_floats(C.byref(p), net, H, C.byref(n)) == 0
            layout, total = synth.net_offsets(i, H, o)
            assert n.value == total and all(off % 4 == 0 for *_, off in layout)
    n = C.c_uint64()
    assert lib.ej_net_floats(C.byref(p), 0, 100, C.byref(n)) == 3      # not a multiple of 32


def test_policy_argument_checks(lib):
    p = N.make_params(E=2, A=10)
    fake = C.c_void_p(4096)
    # misaligned weights and missing outputs are rejected on the host
    assert lib.policy_forward(C.byref(p), fake, 0, 128, 0, C.c_void_p(4100), fake, None, None,
                              None, None, fake, None, None, None) == 1
    assert lib.policy_forward(C.byref(p), fake, 0, 128, 0, fake, fake, None, None,
                              None, None, None, None, None, None) == 1
    assert lib.policy_forward(C.byref(p), fake, 0, 128, 0, fake, fake, None, None,
                              fake, None, fake, None, None, None) == 1   # act without logp
    assert lib.policy_forward(C.byref(p), fake, 7, 128, 0, fake, fake, None, None,
                              None, None, fake, None, None, None) == 1   # unknown network


def test_policy_segmented_shapes(lib):
    """Which network shapes share launches in policy_forward_segments: BF16,
    hidden 128, <= 96 logits, <= 32 inputs (every benchmark network)."""
    from paper_2410_22165_gb300.batch import price_grid
    ok = C.c_int32()
    for levels, n_actions in ((5, 24), (10, 44), (20, 84)):
        p = N.make_params(E=2, A=10, **price_grid(levels))
        assert N.sizes(p).n_actions == n_actions
        for net in (N.NET_POP, N.NET_GOV):
            assert lib.policy_segmented(C.byref(p), net, 128, N.BF16, C.byref(ok)) == 0 and ok.value == 1
            assert lib.policy_segmented(C.byref(p), net, 128, N.FP32, C.byref(ok)) == 0 and ok.value == 0
            assert lib.policy_segmented(C.byref(p), net, 64, N.BF16, C.byref(ok)) == 0 and ok.value == 0
    p = N.make_params(E=2, A=10, **price_grid(30))           # 2 + 2 + 120 = 124 actions: one launch per set
    assert lib.policy_segmented(C.byref(p), N.NET_POP, 128, N.BF16, C.byref(ok)) == 0 and ok.value == 0
    assert lib.policy_segmented(C.byref(p), 7, 128, N.BF16, C.byref(ok)) == 1     # unknown network
    assert lib.policy_segmented(C.byref(p), N.NET_POP, 128, N.BF16, None) == 1    # NULL result


def test_policy_segments_argument_checks(lib):
    p = N.make_params(E=2, A=10)
    fake = C.c_void_p(4096)
    V = C.c_void_p * 1
    one = lambda x: V(x)
    nets = (C.c_int32 * 1)(N.NET_GOV)
    # no sets, NULL arrays, and a mask given for a government set are rejected on the host
    assert lib.policy_forward_segments(0, one(C.addressof(p)), one(fake), nets, one(fake), 128, N.BF16,
                                       one(fake), None, None, None, one(fake), None) == 1
    assert lib.policy_forward_segments(1, None, one(fake), nets, one(fake), 128, N.BF16,
                                       one(fake), None, None, None, one(fake), None) == 1
    assert lib.policy_forward_segments(1, one(C.addressof(p)), one(fake), nets, one(fake), 128, N.BF16,
                                       one(fake), one(fake), None, None, one(fake), None) == 1


def test_rollout_split_argument_checks(lib):
    """Chain counts outside 1..4 and missing buffers are rejected on the host."""
    p = N.make_params(E=4, A=10)
    fake = C.c_void_p(4096)
    buf = N.EjRollout(**{f: 4096 for f, _ in N.EjRollout._fields_})
    for chains in (0, 5, -1):
        assert lib.rollout_split(C.byref(p), fake, 3, 128, N.BF16, fake, fake, C.byref(buf), chains, None) == 1
    assert "chains" in N.load().ej_last_error().decode()
    missing = N.EjRollout(**{f: (0 if f == "rew" else 4096) for f, _ in N.EjRollout._fields_})
    assert lib.rollout_split(C.byref(p), fake, 3, 128, N.BF16, fake, fake, C.byref(missing), 2, None) == 1
    assert lib.rollout_split(C.byref(p), fake, 0, 128, N.BF16, fake, fake, C.byref(buf), 2, None) == 1   # T = 0


@pytest.mark.parametrize("member", [f for f, _ in N.EjRollout._fields_])
def test_ppo_calls_reject_missing_rollout_arrays(lib, member):
    """Every PPO entry point checks the rollout-buffer arrays it reads before
    it enqueues anything: a NULL one returns EJ_ERR_ARG (no GPU is touched)."""
    p = N.make_params(E=2, A=4)
    pp = N.EjPpoParams()
    lib.ej_ppo_params_default(C.byref(pp))
    fake = C.c_void_p(4096)
    T, H = 8, 128
    b = N.EjRollout(**{f: (0 if f == member else 4096) for f, _ in N.EjRollout._fields_})
    gae = member in ("rew", "value", "grew", "gvalue", "done")
    pop_grad = member in ("obs", "mask", "act", "logp", "value")
    gov_grad = member in ("gobs", "gact", "glogp", "gvalue")
    reads = {
        "ppo_advantages": gae,
        "ppo_minibatch_grad pop": pop_grad, "ppo_minibatch_grad gov": gov_grad,
        "ppo_minibatch_grad_global pop": pop_grad, "ppo_minibatch_grad_global gov": gov_grad,
        "ppo_update": gae or pop_grad or gov_grad,
        "ppo_minibatch_grad_static pop": pop_grad or member in ("rew", "value", "done"),
        "ppo_minibatch_grad_static gov": gov_grad or member in ("grew", "gvalue", "done"),
    }
    calls = {
        "ppo_advantages": lambda: lib.ppo_advantages(C.byref(p), C.byref(pp), T, C.byref(b), fake, None),
        "ppo_update": lambda: lib.ppo_update(C.byref(p), C.byref(pp), T, H, N.FP32, fake, fake, fake, fake,
                                             fake, fake, 0, 0, C.byref(b), fake, None, None),
    }
    for net, tag in ((N.NET_POP, "pop"), (N.NET_GOV, "gov")):
        calls[f"ppo_minibatch_grad {tag}"] = lambda net=net: lib.ppo_minibatch_grad(
            C.byref(p), C.byref(pp), T, H, N.FP32, net, fake, C.byref(b), fake, 0, 0, fake, None, None)
        calls[f"ppo_minibatch_grad_global {tag}"] = lambda net=net: lib.ppo_minibatch_grad_global(
            C.byref(p), C.byref(pp), T, H, N.FP32, net, fake, C.byref(b), fake, 0, 0, fake, fake, None, None)
        calls[f"ppo_minibatch_grad_static {tag}"] = lambda net=net: lib.ppo_minibatch_grad_static(
            C.byref(p), C.byref(pp), T, H, N.FP32, net, fake, C.byref(b), 0, 0, fake, None, None)
    for name, call in calls.items():
        if reads[name]:
            assert call() == 1, name
            assert member in lib.ej_last_error().decode(), name


def test_step_host_argument_checks(lib):
    """env_step_host validates on the host: NULL or misaligned workspace, a
    workspace below ej_step_host_workspace_bytes, chunk < 1, draws without
    actions (no GPU is touched)."""
    p = N.make_params(E=2, A=10)
    fake = C.c_void_p(4096)
    need = C.c_uint64()
    assert lib.ej_step_host_workspace_bytes(C.byref(p), 8, C.byref(need)) == 0 and need.value > 0
    assert lib.ej_step_host_workspace_bytes(C.byref(p), 0, C.byref(need)) == 1
    args = lambda ws, nbytes, chunk=8, act=None, gu=None: (
        C.byref(p), fake, 16, chunk, act, None, gu, gu, None, None, None, None, None, None, ws, nbytes, None)
    assert lib.env_step_host(*args(None, 1 << 40)) == 1
    assert lib.env_step_host(*args(C.c_void_p(4100), 1 << 40)) == 1
    lib.ej_step_host_workspace_bytes(C.byref(p), 8, C.byref(need))
    assert lib.env_step_host(*args(fake, need.value - 1)) == 1
    assert "workspace" in lib.ej_last_error().decode()
    assert lib.env_step_host(*args(fake, 1 << 40, chunk=0)) == 1
    assert lib.env_step_host(*args(fake, 1 << 40, gu=fake)) == 1


def test_ppo_minibatches_need_rows(lib):
    """More minibatches than the government network's T x E rows would leave
    some empty: refused on the host (EJ_ERR_ARG) by every PPO entry point,
    starting with the workspace query."""
    pp = N.EjPpoParams()
    lib.ej_ppo_params_default(C.byref(pp))
    p = N.make_params(E=2, A=4)
    nb = C.c_uint64()
    pp.minibatches = 8
    assert lib.ej_ppo_workspace_bytes(C.byref(p), C.byref(pp), 4, 128, C.byref(nb)) == 0       # 8 rows
    assert lib.ej_ppo_workspace_bytes(C.byref(p), C.byref(pp), 3, 128, C.byref(nb)) == 1       # 6 rows
    assert b"minibatches" in lib.ej_last_error()


def test_ppo_hidden_limits(lib):
    """Hidden widths: multiples of 32 up to 256 size a workspace; the BF16
    gradient takes hidden 128 only: refused on the host (EJ_ERR_UNSUPPORTED)."""
    pp = N.EjPpoParams()
    lib.ej_ppo_params_default(C.byref(pp))
    p4 = N.make_params(E=2, A=4, R=4, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=2, gov_enabled=0)
    p12 = N.make_params(E=2, A=4, R=12, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=3, gov_enabled=0)
    nb = C.c_uint64()
    for H in (32, 128, 256):
        assert lib.ej_ppo_workspace_bytes(C.byref(p4), C.byref(pp), 8, H, C.byref(nb)) == 0
    assert lib.ej_ppo_workspace_bytes(C.byref(p4), C.byref(pp), 8, 288, C.byref(nb)) == 3
    assert lib.ej_ppo_workspace_bytes(C.byref(p4), C.byref(pp), 8, 100, C.byref(nb)) == 3
    fake = C.c_void_p(4096)
    b = N.EjRollout(**{f: 4096 for f, _ in N.EjRollout._fields_})
    st = lib.ppo_minibatch_grad(C.byref(p12), C.byref(pp), 8, 256, N.BF16, 0, fake, C.byref(b), fake,
                                0, 0, fake, None, None)
    assert st == 3
    assert lib.ppo_update(C.byref(p12), C.byref(pp), 8, 256, N.BF16, fake, fake, fake, fake, fake, fake, 0, 0,
                          C.byref(b), fake, None, None) == 3
