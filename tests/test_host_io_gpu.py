"""env_step_host (the C ABI's host-buffer env_step, pipelined in chunks) against
the device path: same outputs bit for bit, with a ragged last chunk, the state
continuing across calls, in-kernel draws and a subset of the outputs."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def test_step_host_equals_device_steps():
    import paper_2410_22165_gb300 as P
    E, A, n = 8, 10, 250
    kw = dict(T_ep=30, T_tax=6)
    ref, got = P.VecEnv(E, A, **kw), P.VecEnv(E, A, **kw)
    ref.reset(seed=3)
    got.reset(seed=3)
    d = ref.fill_draws(seed=3, g0=0, n_steps=2 * n)
    out_ref = ref.step(2 * n, act=d["act"], gov_act=d["gov_act"], gather_u=d["gather_u"], tb=d["tb"])
    host_in = {k: v.cpu().pin_memory() for k, v in d.items()}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out_ref.items()}
    for half in range(2):                       # two calls: the state carries over
        sl = slice(half * n, (half + 1) * n)
        got.step_host(n, {k: v[sl] for k, v in host_in.items()}, {k: v[sl] for k, v in host_out.items()},
                      chunk=64)
    for k, v in out_ref.items():
        assert torch.equal(host_out[k], v.cpu()), k
    # state: every field, the order book up to its live length (slots past it are unused)
    for name in ("coin", "esc", "income", "uprev", "nord", "counts", "sc", "inv", "inve", "sg", "t", "gstep",
                 "episode", "pop", "rates", "ugprev", "level_count"):
        assert torch.equal(got.field(name), ref.field(name)), name
    live = ref.field("level_count").sum(1)
    for e in range(E):
        nb = int(live[e])
        assert torch.equal(got.field("book")[e, :nb], ref.field("book")[e, :nb])


def test_step_host_kernel_draws_and_output_subset():
    """No host inputs (the kernel draws actions and rate levels itself), only
    rewards and masks copied back; one chunk larger than the call."""
    import paper_2410_22165_gb300 as P
    E, A, n = 5, 37, 90
    kw = dict(T_ep=40, T_tax=9)
    ref, got = P.VecEnv(E, A, **kw), P.VecEnv(E, A, **kw)
    ref.reset(seed=9)
    got.reset(seed=9)
    out_ref = ref.step(n)
    host_out = {k: torch.empty(out_ref[k].shape, dtype=out_ref[k].dtype).pin_memory() for k in ("rew", "mask")}
    got.step_host(n, {}, host_out, chunk=500)
    for k, v in host_out.items():
        assert torch.equal(v, out_ref[k].cpu()), k
    assert torch.equal(got.field("coin"), ref.field("coin"))


def test_step_host_rejects_small_workspace():
    import ctypes as C
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    env = P.VecEnv(2, 10)
    env.reset(seed=0)
    nbytes = C.c_uint64()
    assert N.load().ej_step_host_workspace_bytes(C.byref(env.p), 10, C.byref(nbytes)) == 0
    ws = torch.empty(int(nbytes.value) - 256, dtype=torch.uint8, device=env.device)
    st = N.load().env_step_host(C.byref(env.p), C.c_void_p(env.state.data_ptr()), 10, 10, None, None, None, None,
                                None, None, None, None, None, None, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert st == 1 and "workspace" in N.load().ej_last_error().decode()
