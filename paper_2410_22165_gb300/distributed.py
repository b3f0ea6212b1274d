"""Data-parallel PPO update over the ranks of a torch.distributed group.

Each rank runs its own environments and rollout (the environment step and the
rollout shard over environments with no exchange).  The PPO update of Section
4 has one exchange step: per minibatch and network, the loss is taken over the
union of the ranks' minibatch rows, so

  1. each rank computes the moments of its minibatch's GAE advantages
     {rows, sum, sum of squares} and the ranks sum them (all-reduce), which
     gives every rank the normalisation of the union minibatch;
  2. each rank computes its part of the union minibatch's gradient with those
     moments, and the ranks sum the gradients (all-reduce);
  3. every rank takes the same Adam step with the summed gradient, so the
     weights stay identical on all ranks.

The order of minibatches, networks and Adam steps is that of the library's
own single-process ppo_update (population, then government, per minibatch).
The per-rank work goes through an `ops` object; the default one calls the
library (PPO.minibatch_moments, PPO.minibatch_grad with moments, PPO.adam).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import _native as N


class LibraryOps:
    """The per-rank steps of the update, on the GPU through the C ABI."""

    def __init__(self, ppo):
        self.ppo = ppo

    def advantages(self, rollout):
        self.ppo.advantages(rollout)

    def moments(self, rollout, net, ctr, mb):
        return self.ppo.minibatch_moments(rollout, net, ctr, mb)

    def grad(self, rollout, net, ctr, mb, moments):
        return self.ppo.minibatch_grad(rollout, net, ctr, mb, moments=moments)

    def adam(self, net, grad, step):
        self.ppo.adam(net, grad, step)

    def params(self):
        pp = self.ppo.pp
        return pp.epochs, pp.minibatches


class DistributedPPO:
    """PPO updates whose minibatch statistics and gradients are summed over
    the ranks of `group` (None: the default group).  With one rank it
    computes exactly what PPO.update computes."""

    def __init__(self, ppo=None, group=None, ops=None):
        if ops is None and ppo is None:
            raise ValueError("give a PPO object or an ops object")
        self.ops = ops if ops is not None else LibraryOps(ppo)
        self.group = group
        self.adam_steps = 0
        self.updates = 0

    def _sum(self, t):
        # over the group whenever one is initialised (with one rank an identity
        # that still goes through the backend, e.g. NCCL on the device)
        if dist.is_available() and dist.is_initialized():
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def update(self, rollout):
        """One update; returns the per-network loss sums over all ranks and
        minibatches (float64 [2][8], the ppo_minibatch_grad statistics)."""
        epochs, minibatches = self.ops.params()
        self.ops.advantages(rollout)
        totals = None
        step = self.adam_steps
        for ep in range(epochs):
            ctr = (self.updates * epochs + ep) & 0xFFFFFFFF
            for mb in range(minibatches):
                step += 1
                for net in (N.NET_POP, N.NET_GOV):
                    c = ctr ^ (0x80000000 if net == N.NET_GOV else 0)
                    m = self._sum(self.ops.moments(rollout, net, c, mb))
                    g, st = self.ops.grad(rollout, net, c, mb, m)
                    self._sum(g)
                    self.ops.adam(net, g, step)
                    st = self._sum(st.clone())
                    if totals is None:
                        totals = torch.zeros((2,) + tuple(st.shape), dtype=st.dtype, device=st.device)
                    totals[net] += st
        self.adam_steps = step
        self.updates += 1
        return totals
