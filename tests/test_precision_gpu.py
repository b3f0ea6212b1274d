"""Error of BF16 and FP32 values, advantages and returns against float64.

One rollout (BF16 policy, 16 environments x 20 agents x 64 steps) fixes the
trajectory: rewards, episode ends and observations.  The critic is evaluated
on every observation of the rollout by the library's BF16 and FP32 forward
kernels and by the float64 oracle; GAE (gamma 0.99, lambda 0.95) turns each
set of values into advantages and returns.  The errors relative to the
float64 results (L2 norm over all rows and steps, over the L2 norm of the
float64 quantity) are printed and bounded:

  FP32: values, advantages, returns within 1e-5;
  BF16: values and returns within 2e-2, advantages within 2e-1 (an advantage
        is a difference of returns and values, so it keeps their absolute
        error with a smaller magnitude).

The environment arithmetic is the same in both forms (integer state
bit-exact, float decisions in float32), so the BF16 form changes only these.
"""
import numpy as np
import pytest

import synth
from oracle import policy as op
from oracle import ppo as oppo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_22165_gb300 import build
    build.build()


def test_value_advantage_return_errors_against_float64():
    import paper_2410_22165_gb300 as P
    from paper_2410_22165_gb300 import _native as N
    E, A, T = 16, 20, 64
    env = P.VecEnv(E, A, T_ep=40, T_tax=10)
    pw = synth.net_weights(9, 0, env.D, H, env.nA)
    gw = synth.net_weights(9, 1, env.G, H, env.p.nb * env.p.tax_levels)
    pol = {prec: P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H, precision=prec)
           for prec in ("bf16", "fp32")}
    ro = P.Rollout(env, pol["bf16"], T)
    ro.reset(seed=9)
    ro.run()
    obs = ro.buf["obs"]                                    # [T+1][E][A][D]
    rew = ro.buf["rew"].double().cpu().numpy().reshape(T, E * A)
    done = np.repeat(ro.buf["done"].cpu().numpy()[:, :, None], A, axis=2).reshape(T, E * A)
    values = {}
    for prec, p in pol.items():
        v = [p.forward(N.NET_POP, obs[t].contiguous(), sample=False)["value"] for t in range(T + 1)]
        values[prec] = torch.stack(v).double().cpu().numpy()
    w64 = synth.unpack(pw, env.D, H, env.nA)
    x = obs.double().cpu().numpy().reshape((T + 1) * E * A, env.D)
    values["f64"] = op.mlp64(w64, x)[1].reshape(T + 1, E * A)
    res = {k: oppo.gae64(rew, values[k], done, 0.99, 0.95) for k in values}
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    err = {}
    for prec in ("bf16", "fp32"):
        err[prec] = dict(value=rel(values[prec], values["f64"]), adv=rel(res[prec][0], res["f64"][0]),
                         ret=rel(res[prec][1], res["f64"][1]))
    print("relative L2 error against float64:", err)
    assert max(err["fp32"].values()) <= 1e-5
    assert err["bf16"]["value"] <= 2e-2 and err["bf16"]["ret"] <= 2e-2 and err["bf16"]["adv"] <= 2e-1
