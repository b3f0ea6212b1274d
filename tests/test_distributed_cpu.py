"""The data-parallel PPO update (DistributedPPO) on two gloo ranks on the CPU.

The per-rank steps (minibatch rows, advantage moments, gradient, Adam) come
from the float64 oracle here, standing in for the library's GPU kernels; what
is tested is the orchestration: the two all-reduces per minibatch and network,
the order of minibatches, networks and Adam steps, and that both ranks end
with identical weights equal to a single-process update whose every
minibatch is the union of the ranks' minibatches.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import ppo as oppo  # noqa: E402
from synth import shuffle  # noqa: E402

IN, H, O = 5, 8, 6
EPOCHS, MINIBATCHES, SEED = 2, 3, 17
COEF = dict(clip=0.2, vf_coef=0.25, vclip=10.0, ent_coef=0.1)
NAMES = ["W1", "b1", "W2", "b2", "W3", "b3", "V1", "c1", "V2", "c2", "V3", "c3"]


def _rank_data(rank, net):
    """A synthetic rollout slice of one rank and network (rows differ per rank)."""
    rng = np.random.default_rng(1000 * rank + net)
    N = 30 + 7 * rank + 3 * net
    valid = rng.random((N, O)) < 0.7
    valid[:, 0] = True
    act = np.array([rng.choice(np.nonzero(v)[0]) for v in valid])[:, None]
    return dict(x=rng.normal(size=(N, IN)), act=act, valid=valid, lpo=rng.normal(size=N) * 0.3 - 1.5,
                vo=rng.normal(size=N), adv=rng.normal(size=N), ret=rng.normal(size=N) * 2)


def _init_weights(net):
    rng = np.random.default_rng(77 + net)
    shapes = dict(W1=(IN, H), b1=(H,), W2=(H, H), b2=(H,), W3=(H, O), b3=(O,), V1=(IN, H), c1=(H,),
                  V2=(H, H), c2=(H,), V3=(H, 1), c3=(1,))
    return {k: rng.normal(size=shapes[k]) * 0.4 for k in NAMES}


def _flat(g):
    return np.concatenate([np.asarray(g[k], np.float64).ravel() for k in NAMES])


def _unflat(v, like):
    out, p = {}, 0
    for k in NAMES:
        n = like[k].size
        out[k] = v[p:p + n].reshape(like[k].shape)
        p += n
    return out


class OracleOps:
    """Per-rank steps of the update in float64 (the test's stand-in for the GPU kernels)."""

    def __init__(self, rank):
        self.data = [_rank_data(rank, 0), _rank_data(rank, 1)]
        self.w = [_init_weights(0), _init_weights(1)]
        self.m = [np.zeros_like(_flat(self.w[n])) for n in (0, 1)]
        self.v = [np.zeros_like(_flat(self.w[n])) for n in (0, 1)]

    def params(self):
        return EPOCHS, MINIBATCHES

    def advantages(self, rollout):
        pass

    def _rows(self, net, ctr, mb):
        return shuffle.minibatch_rows(mb, MINIBATCHES, len(self.data[net]["adv"]), SEED, ctr)

    def moments(self, rollout, net, ctr, mb):
        a = self.data[net]["adv"][self._rows(net, ctr, mb)]
        return torch.tensor([len(a), a.sum(), (a * a).sum()], dtype=torch.float64)

    def grad(self, rollout, net, ctr, mb, moments):
        d, r = self.data[net], self._rows(net, ctr, mb)
        loss, g, st = oppo.ppo_loss_grad64(self.w[net], d["x"][r], d["act"][r], d["valid"][r], d["lpo"][r],
                                           d["vo"][r], d["adv"][r], d["ret"][r], heads=1, head=O,
                                           moments=moments.numpy(), **COEF)
        stats = torch.zeros(8, dtype=torch.float64)
        stats[2] = loss
        return torch.from_numpy(_flat(g)), stats

    def adam(self, net, grad, step):
        w = _flat(self.w[net])
        w, self.m[net], self.v[net] = oppo.adam64(w, grad.numpy(), self.m[net], self.v[net], step, lr=1e-2)
        self.w[net] = _unflat(w, self.w[net])


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2410_22165_gb300.distributed import DistributedPPO
        ops = OracleOps(rank)
        dppo = DistributedPPO(ops=ops)
        totals = [dppo.update(None) for _ in range(2)]
        np.save(os.path.join(out, f"w{rank}.npy"),
                np.concatenate([_flat(ops.w[0]), _flat(ops.w[1]), totals[-1].numpy().ravel()]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _single_process_reference(world, updates):
    """Every minibatch = the union of the ranks' minibatches, one process."""
    data = [[_rank_data(r, n) for n in (0, 1)] for r in range(world)]
    w = [_init_weights(0), _init_weights(1)]
    m = [np.zeros_like(_flat(w[n])) for n in (0, 1)]
    v = [np.zeros_like(_flat(w[n])) for n in (0, 1)]
    step = 0
    for u in range(updates):
        for ep in range(EPOCHS):
            ctr = u * EPOCHS + ep
            for mb in range(MINIBATCHES):
                step += 1
                for net in (0, 1):
                    c = ctr ^ (0x80000000 if net == 1 else 0)
                    parts = [data[r][net] for r in range(world)]
                    rows = [shuffle.minibatch_rows(mb, MINIBATCHES, len(p["adv"]), SEED, c) for p in parts]
                    cat = {k: np.concatenate([p[k][rr] for p, rr in zip(parts, rows)]) for k in parts[0]}
                    _, g, _ = oppo.ppo_loss_grad64(w[net], cat["x"], cat["act"], cat["valid"], cat["lpo"],
                                                   cat["vo"], cat["adv"], cat["ret"], heads=1, head=O, **COEF)
                    flat, m[net], v[net] = oppo.adam64(_flat(w[net]), _flat(g), m[net], v[net], step, lr=1e-2)
                    w[net] = _unflat(flat, w[net])
    return np.concatenate([_flat(w[0]), _flat(w[1])])


def test_two_ranks_match_union_minibatch_update(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [np.load(os.path.join(tmp_path, f"w{r}.npy")) for r in range(world)]
    nw = len(_single_process_reference(1, 0))
    assert np.array_equal(got[0], got[1]), "ranks diverged"
    ref = _single_process_reference(world, 2)
    assert np.allclose(got[0][:nw], ref, rtol=1e-10, atol=1e-12)
    assert np.all(np.isfinite(got[0][nw:]))


def test_one_rank_without_process_group_is_plain_update():
    """No process group: DistributedPPO is the single-process update of its own rows."""
    from paper_2410_22165_gb300.distributed import DistributedPPO
    ops = OracleOps(0)
    DistributedPPO(ops=ops).update(None)
    got = np.concatenate([_flat(ops.w[0]), _flat(ops.w[1])])
    data = [_rank_data(0, n) for n in (0, 1)]
    w = [_init_weights(0), _init_weights(1)]
    m = [np.zeros_like(_flat(w[n])) for n in (0, 1)]
    v = [np.zeros_like(_flat(w[n])) for n in (0, 1)]
    step = 0
    for ep in range(EPOCHS):
        for mb in range(MINIBATCHES):
            step += 1
            for net in (0, 1):
                c = ep ^ (0x80000000 if net == 1 else 0)
                d = data[net]
                r = shuffle.minibatch_rows(mb, MINIBATCHES, len(d["adv"]), SEED, c)
                _, g, _ = oppo.ppo_loss_grad64(w[net], d["x"][r], d["act"][r], d["valid"][r], d["lpo"][r],
                                               d["vo"][r], d["adv"][r], d["ret"][r], heads=1, head=O, **COEF)
                flat, m[net], v[net] = oppo.adam64(_flat(w[net]), _flat(g), m[net], v[net], step, lr=1e-2)
                w[net] = _unflat(flat, w[net])
    assert np.allclose(got, np.concatenate([_flat(w[0]), _flat(w[1])]), rtol=1e-10, atol=1e-12)
