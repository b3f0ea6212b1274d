"""Kernel side of the data-parallel PPO update, on one GPU.

Two rollouts of different environments stand in for two ranks: their
minibatch advantage moments are summed, each computes its part of the
gradient with the summed moments (ppo_minibatch_grad_global), and the sum of
the parts is compared with the oracle's gradient of the union minibatch
(float32 path: float64 oracle; BF16 path: the oracle's BF16-operand form).
DistributedPPO without a process group reproduces PPO.update.
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


def _rank(seed, precision, E=2, A=4, T=16):
    import paper_2410_22165_gb300 as P
    env = P.VecEnv(E, A, T_ep=12, T_tax=4)
    pw = synth.net_weights(5, 0, env.D, H, env.nA)
    gw = synth.net_weights(5, 1, env.G, H, env.p.nb * env.p.tax_levels)
    pol = P.Policy(env, torch.from_numpy(pw), torch.from_numpy(gw), hidden=H)
    ro = P.Rollout(env, pol, T)
    ro.reset(seed=seed)
    ro.run()
    ppo = P.PPO(pol, T, precision=precision, minibatches=4, seed=77)
    ppo.advantages(ro)
    return env, ro, ppo, pw, gw


def _rows_inputs(env, ro, ppo, net, rows):
    b = {k: v.cpu().numpy() for k, v in ro.buf.items()}
    E, A, T = env.E, env.A, ro.T
    if net == 0:
        done = np.repeat(b["done"][:, :, None], A, axis=2).reshape(T, E * A)
        adv, ret = oppo.gae64(b["rew"].reshape(T, E * A), b["value"].reshape(T + 1, E * A), done,
                              ppo.pp.gamma, ppo.pp.lam)
        return dict(x=b["obs"][:T].reshape(T * E * A, env.D)[rows],
                    valid=op.mask_bits(b["mask"][:T].reshape(T * E * A, env.W).view(np.uint32), env.nA)[rows],
                    act=b["act"].reshape(-1, 1)[rows], lpo=b["logp"].reshape(-1)[rows],
                    vo=b["value"][:T].reshape(-1)[rows], adv=adv.reshape(-1)[rows], ret=ret.reshape(-1)[rows])
    adv, ret = oppo.gae64(b["grew"], b["gvalue"], b["done"], ppo.pp.gamma, ppo.pp.lam)
    L = env.p.tax_levels
    return dict(x=b["gobs"][:T].reshape(T * E, env.G)[rows], valid=np.ones((len(rows), env.p.nb * L), bool),
                act=b["gact"].reshape(T * E, env.p.nb)[rows], lpo=b["glogp"].reshape(-1)[rows],
                vo=b["gvalue"][:T].reshape(-1)[rows], adv=adv.reshape(-1)[rows], ret=ret.reshape(-1)[rows])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("net", [0, 1])
def test_two_rank_parts_sum_to_union_gradient(precision, net):
    ranks = [_rank(seed, precision, E=2 if net == 0 else 8) for seed in (11, 12)]
    ctr, mb = 3, 1
    moments = sum(r[2].minibatch_moments(r[1], net, ctr, mb) for r in ranks)
    grad = sum(r[2].minibatch_grad(r[1], net, ctr, mb, moments=moments)[0] for r in ranks).cpu().numpy()
    parts = []
    for env, ro, ppo, pw, gw in ranks:
        N = ro.T * (env.E * env.A if net == 0 else env.E)
        parts.append(_rows_inputs(env, ro, ppo, net, shuffle.minibatch_rows(mb, 4, N, 77, ctr)))
    cat = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    assert float(moments[0]) == len(cat["adv"])
    env, ro, ppo, pw, gw = ranks[0]
    in_dim = env.D if net == 0 else env.G
    O = env.nA if net == 0 else env.p.nb * env.p.tax_levels
    heads, head = (1, env.nA) if net == 0 else (env.p.nb, env.p.tax_levels)
    w = synth.unpack(pw if net == 0 else gw, in_dim, H, O)
    _, ref, _ = oppo.ppo_loss_grad64(w, cat["x"], cat["act"], cat["valid"], cat["lpo"], cat["vo"], cat["adv"],
                                     cat["ret"], clip=ppo.pp.clip, vf_coef=ppo.pp.vf_coef, vclip=ppo.pp.vclip,
                                     ent_coef=ppo.pp.ent_coef, heads=heads, head=head,
                                     operand=oppo.bf16_round if precision == "bf16" else None)
    got = synth.unpack(grad, in_dim, H, O)
    tol = 1e-3 if precision == "fp32" else 1e-2
    for k, r in ref.items():
        assert np.max(np.abs(got[k].reshape(r.shape) - r)) <= tol * np.abs(r).max() + 1e-7, k


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_distributed_update_without_group_equals_update(precision):
    from paper_2410_22165_gb300.distributed import DistributedPPO
    _, ro1, ppo1, _, _ = _rank(21, precision)
    _, ro2, ppo2, _, _ = _rank(21, precision)
    ppo1.update(ro1)
    DistributedPPO(ppo2).update(ro2)
    for a, b in ((ppo1.policy.pop_w, ppo2.policy.pop_w), (ppo1.policy.gov_w, ppo2.policy.gov_w)):
        # the advantage sums are double atomics (order not fixed): equal up to their last bits
        assert torch.allclose(a, b, rtol=0, atol=1e-7)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_nccl_one_rank_update_equals_update(precision):
    """The update through a real NCCL process group (one rank on this GPU: the
    all-reduces of the moments and gradients run on the device and sum one
    part) equals PPO.update."""
    import socket
    import torch.distributed as dist
    from paper_2410_22165_gb300.distributed import DistributedPPO
    if not dist.is_available() or not dist.is_nccl_available():
        pytest.skip("no NCCL")
    import os
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")     # no NVLink multicast objects
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        _, ro1, ppo1, _, _ = _rank(23, precision)
        _, ro2, ppo2, _, _ = _rank(23, precision)
        ppo1.update(ro1)
        DistributedPPO(ppo2).update(ro2)
        torch.cuda.synchronize()
        for a, b in ((ppo1.policy.pop_w, ppo2.policy.pop_w), (ppo1.policy.gov_w, ppo2.policy.gov_w)):
            assert torch.allclose(a, b, rtol=0, atol=1e-7)
    finally:
        dist.destroy_process_group()
