"""The PPO minibatch gradient without a workspace (ppo_minibatch_grad_static).

Some callers of this library cannot allocate device memory: hosts whose
device memory belongs to another runtime's pool allocator, C programs without
a device allocator of their own, and service loops that must not allocate
once running.  For them the library offers an entry point
whose scratch is a static device array it holds itself.  This file checks,
through the C ABI, that two calls in a row give the gradient of the
workspace-based entry point, within the gradient tolerance the other PPO tests
use (1e-3 of the largest entry of each tensor), and that sizes beyond the
array's capacity are refused before anything runs.  It is named so that pytest
collects it after every other test file.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def _setup(E, A, T, seed, **kw):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, **kw)
    pw = synth.net_weights(seed, 0, env.D, H, env.nA)
    gw = synth.net_weights(seed, 1, env.G, H, env.p.nb * env.p.tax_levels)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=seed)
    ro.run()
    ppo = P.PPO(pol, T, minibatches=4, seed=77)
    return env, pol, ro, ppo


def _static_grad(env, pol, ro, ppo, net, ctr, mb):
    """One call through the C ABI; returns the gradient, the statistics and
    the device memory torch holds after the call minus before it (the
    outputs are allocated before the measurement)."""
    from paper_2410_22165_gb300 import _native as N
    w = pol.pop_w if net == 0 else pol.gov_w
    grad = torch.full_like(w, float("nan"))
    stats = torch.empty(8, dtype=torch.float64, device=w.device)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    st = N.load().ppo_minibatch_grad_static(
        C.byref(env.p), C.byref(ppo.pp), ppo.T, H, N.FP32, net, C.c_void_p(w.data_ptr()), C.byref(ro._c),
        ctr, mb, C.c_void_p(grad.data_ptr()), C.c_void_p(stats.data_ptr()),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st, "ppo_minibatch_grad_static")
    torch.cuda.synchronize()
    return grad, stats, torch.cuda.memory_allocated() - before


@pytest.mark.parametrize("net", [0, 1])
def test_static_scratch_gradient_equals_workspace_gradient(net):
    E, A, T = (2, 4, 16) if net == 0 else (8, 4, 16)
    env, pol, ro, ppo = _setup(E, A, T, seed=2, T_ep=12, T_tax=4)
    ppo.advantages(ro)
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
    for ctr, mb in ((3, 1), (4, 2)):                     # two calls in a row
        g_static, s_static, grown = _static_grad(env, pol, ro, ppo, net, ctr, mb)
        assert grown == 0                                  # the call itself allocates nothing
        g_ws, s_ws = ppo.minibatch_grad(ro, net, ctr, mb)
        torch.cuda.synchronize()
        a = synth.unpack(g_static.cpu().numpy(), in_dim, H, O)
        b = synth.unpack(g_ws.cpu().numpy(), in_dim, H, O)
        for k in b:
            tol = 1e-3 * np.abs(b[k]).max() + 1e-7
            assert np.max(np.abs(a[k] - b[k])) <= tol, (ctr, mb, k)
        assert not torch.isnan(g_static).any()
        assert torch.allclose(s_static, s_ws, rtol=1e-5, atol=1e-9)


def test_sizes_beyond_the_static_array_are_refused():
    from paper_2410_22165_gb300 import _native as N
    p = N.make_params(E=1024, A=100)
    pp = N.EjPpoParams()
    N.load().ej_ppo_params_default(C.byref(pp))
    rollout = N.EjRollout()
    st = N.load().ppo_minibatch_grad_static(C.byref(p), C.byref(pp), 128, H, N.FP32, 0, C.c_void_p(4096),
                                            C.byref(rollout), 0, 0, C.c_void_p(4096), None, None)
    assert st == 3
    assert "static" in N.load().ej_last_error().decode()


def test_bf16_is_refused():
    """The static entry point computes in FP32 only."""
    from paper_2410_22165_gb300 import _native as N
    p = N.make_params(E=2, A=4)
    pp = N.EjPpoParams()
    N.load().ej_ppo_params_default(C.byref(pp))
    rollout = N.EjRollout(**{f: 4096 for f, _ in N.EjRollout._fields_})
    st = N.load().ppo_minibatch_grad_static(C.byref(p), C.byref(pp), 16, H, N.BF16, 0, C.c_void_p(4096),
                                            C.byref(rollout), 0, 0, C.c_void_p(4096), None, None)
    assert st == 3
