"""PPO update on the GPU (thin wrapper of the C ABI)."""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .env import _ptr, _stream
from .policy import Policy, Rollout


class PPO:
    """Adam state, workspace and the update calls for a Policy and its rollouts."""

    def __init__(self, policy: Policy, T: int, precision: str = "fp32", **overrides):
        """precision of the update's GEMMs (independent of the policy's
        forward precision used by rollouts)."""
        from .policy import PRECISION
        self.policy, self.env, self.T = policy, policy.env, T
        self.precision = PRECISION[precision]
        self.pp = N.EjPpoParams()
        N.check(N.load().ej_ppo_params_default(C.byref(self.pp)), "ej_ppo_params_default")
        for k, v in overrides.items():
            if not hasattr(self.pp, k):
                raise KeyError(k)
            setattr(self.pp, k, v)
        nbytes = C.c_uint64()
        self.layout = policy.layout
        N.check(N.load().ej_ppo_workspace_bytes_agents(C.byref(self.env.p), C.byref(self.pp), T, policy.hidden,
                                                       self.layout, C.byref(nbytes)), "ej_ppo_workspace_bytes_agents")
        dev = self.env.device
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
        self.m = [torch.zeros_like(policy.pop_w), torch.zeros_like(policy.gov_w)]
        self.v = [torch.zeros_like(policy.pop_w), torch.zeros_like(policy.gov_w)]
        self.adam_steps = 0
        self.updates = 0

    def offsets(self):
        off = (C.c_uint64 * 4)()
        N.check(N.load().ej_ppo_workspace_offsets(C.byref(self.env.p), C.byref(self.pp), self.T,
                                                  self.policy.hidden, off), "ej_ppo_workspace_offsets")
        return list(off)

    def advantages(self, rollout: Rollout, stream=None):
        N.check(N.load().ppo_advantages(C.byref(self.env.p), C.byref(self.pp), self.T, C.byref(rollout._c),
                                        _ptr(self.workspace), _stream(stream)), "ppo_advantages")
        E, A, T = self.env.E, self.env.A, self.T
        o = self.offsets()
        ws = self.workspace
        view = lambda off, n: ws[off: off + 4 * n].view(torch.float32)
        return dict(adv=view(o[0], T * E * A).view(T, E, A), ret=view(o[1], T * E * A).view(T, E, A),
                    gadv=view(o[2], T * E).view(T, E), gret=view(o[3], T * E).view(T, E))

    def minibatch_rows(self, net: int, minibatch: int) -> int:
        """Rows of minibatch `minibatch` (floor((m+1)N/M) - floor(mN/M)); for
        per-agent population networks, A times the positions of the T x E
        (step, environment) permutation."""
        M = self.pp.minibatches
        if net == N.NET_POP and self.layout != N.NETS_SHARED:
            n = self.T * self.env.E
            return self.env.A * ((minibatch + 1) * n // M - minibatch * n // M)
        n = self.T * (self.env.E * self.env.A if net == N.NET_POP else self.env.E)
        return (minibatch + 1) * n // M - minibatch * n // M

    def minibatch_moments(self, rollout: Rollout, net: int, shuffle_ctr: int, minibatch: int, stream=None):
        """{rows, sum, sum of squares} of this minibatch's advantages (device float64[3])."""
        m = torch.empty(3, dtype=torch.float64, device=self.env.device)
        N.check(N.load().ppo_minibatch_moments(C.byref(self.env.p), C.byref(self.pp), self.T, net,
                                               C.byref(rollout._c), _ptr(self.workspace), shuffle_ctr, minibatch,
                                               _ptr(m), _stream(stream)), "ppo_minibatch_moments")
        return m

    def minibatch_grad(self, rollout: Rollout, net: int, shuffle_ctr: int, minibatch: int, stream=None,
                       weights: torch.Tensor | None = None, moments: torch.Tensor | None = None):
        """Gradient of one minibatch's loss (and the loss sums, float64[8]);
        `weights` defaults to the policy's current vector of `net`.  With
        `moments` (device float64[3], summed over the ranks of a data-parallel
        update) it is this rank's part of the union minibatch's gradient."""
        pol = self.policy
        w = weights if weights is not None else (pol.pop_w if net == N.NET_POP else pol.gov_w)
        w = w.contiguous()
        grad = torch.empty_like(w)
        stats = torch.empty(8, dtype=torch.float64, device=w.device)
        lib = N.load()
        if net == N.NET_POP and self.layout != N.NETS_SHARED:
            if moments is not None:
                raise NotImplementedError("data-parallel moments with per-agent networks")
            N.check(lib.ppo_minibatch_grad_agents(C.byref(self.env.p), C.byref(self.pp), self.T, pol.hidden,
                                                  self.precision, self.layout, _ptr(w), C.byref(rollout._c),
                                                  _ptr(self.workspace), shuffle_ctr, minibatch, _ptr(grad),
                                                  _ptr(stats), _stream(stream)), "ppo_minibatch_grad_agents")
        elif moments is None:
            N.check(lib.ppo_minibatch_grad(C.byref(self.env.p), C.byref(self.pp), self.T, pol.hidden,
                                           self.precision, net, _ptr(w), C.byref(rollout._c),
                                           _ptr(self.workspace), shuffle_ctr, minibatch, _ptr(grad),
                                           _ptr(stats), _stream(stream)), "ppo_minibatch_grad")
        else:
            moments = moments.to(torch.float64).contiguous()
            N.check(lib.ppo_minibatch_grad_global(C.byref(self.env.p), C.byref(self.pp), self.T, pol.hidden,
                                                  self.precision, net, _ptr(w), C.byref(rollout._c),
                                                  _ptr(self.workspace), shuffle_ctr, minibatch, _ptr(moments),
                                                  _ptr(grad), _ptr(stats), _stream(stream)),
                    "ppo_minibatch_grad_global")
        return grad, stats

    def adam(self, net: int, grad: torch.Tensor, step: int, stream=None):
        """One Adam step of network `net` with the given gradient (step counts from 1)."""
        pol, pp = self.policy, self.pp
        w = pol.pop_w if net == N.NET_POP else pol.gov_w
        N.check(N.load().adam_step(w.numel(), _ptr(w), _ptr(grad), _ptr(self.m[net]), _ptr(self.v[net]), step,
                                   pp.lr, pp.beta1, pp.beta2, pp.eps, _stream(stream)), "adam_step")

    def loss(self, weights: torch.Tensor, rollout: Rollout, net: int, shuffle_ctr: int, minibatch: int):
        """Differentiable minibatch loss: forward and backward are the library's
        hand-written kernels (see PPOLoss)."""
        return PPOLoss.apply(weights, self, rollout, net, shuffle_ctr, minibatch)

    def update(self, rollout: Rollout, stream=None):
        pol = self.policy
        stats = torch.empty((2, 8), dtype=torch.float32, device=pol.pop_w.device)
        N.check(N.load().ppo_update_agents(C.byref(self.env.p), C.byref(self.pp), self.T, pol.hidden, self.precision,
                                           self.layout, _ptr(pol.pop_w), _ptr(pol.gov_w), _ptr(self.m[0]),
                                           _ptr(self.v[0]), _ptr(self.m[1]), _ptr(self.v[1]), self.adam_steps,
                                           self.updates, C.byref(rollout._c), _ptr(self.workspace), _ptr(stats),
                                           _stream(stream)), "ppo_update_agents")
        self.adam_steps += self.pp.epochs * self.pp.minibatches
        self.updates += 1
        return stats


class PPOLoss(torch.autograd.Function):
    """Clipped PPO loss of one minibatch (Section 4) as a torch autograd node.

    forward: one ppo_minibatch_grad call, which runs actor and critic forward,
    the loss and the hand-written backward in the library's kernels and
    returns the minibatch's loss (float64, entry 7 of its statistics).
    backward: the saved gradient scaled by the incoming gradient.  The advantages come from
    the last PPO.advantages call, as for ppo_minibatch_grad.
    """

    @staticmethod
    def forward(ctx, weights, ppo, rollout, net, shuffle_ctr, minibatch):
        grad, stats = ppo.minibatch_grad(rollout, net, shuffle_ctr, minibatch, weights=weights.detach())
        ctx.save_for_backward(grad)
        return stats[7].to(weights.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None
