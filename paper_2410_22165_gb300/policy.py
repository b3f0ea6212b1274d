"""Policy forward, sampling and rollouts on the GPU (thin wrappers of the C ABI)."""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .env import VecEnv, _ptr, _stream

PRECISION = {"fp32": N.FP32, "bf16": N.BF16}
LAYOUT = {"shared": N.NETS_SHARED, "independent": N.NETS_INDEPENDENT, "ctde": N.NETS_CTDE}


class Policy:
    """Population and government actor/critic weights (device, float32 vectors
    in the documented layout) and their forward pass.  layout (Section 5):
    "shared" (one population network), "independent" (an actor and a critic
    per agent) or "ctde" (an actor per agent, one critic); per-agent weights
    are A vectors, [A * n_pop] floats."""

    def __init__(self, env: VecEnv, pop_weights: torch.Tensor, gov_weights: torch.Tensor,
                 hidden: int = 128, precision: str = "fp32", layout: str = "shared"):
        self.env = env
        self.hidden = hidden
        self.precision = PRECISION[precision]
        self.layout = LAYOUT[layout]
        self.n_pop = self.net_floats(env, N.NET_POP, hidden)
        self.n_gov = self.net_floats(env, N.NET_GOV, hidden)
        self.pop_w = pop_weights.to(env.device, torch.float32).contiguous()
        self.gov_w = gov_weights.to(env.device, torch.float32).contiguous()
        groups = 1 if self.layout == N.NETS_SHARED else env.A
        assert self.pop_w.numel() == self.n_pop * groups and self.gov_w.numel() == self.n_gov

    @staticmethod
    def net_floats(env, net, hidden):
        n = C.c_uint64()
        N.check(N.load().ej_net_floats(C.byref(env.p), net, hidden, C.byref(n)), "ej_net_floats")
        return n.value

    def forward(self, net, obs, mask=None, u=None, sample=True, logits=False, entropy=False,
                stream=None):
        env = self.env
        dev = env.device
        rows = env.E * env.A if net == N.NET_POP else env.E
        heads = 1 if net == N.NET_POP else env.p.nb
        O = env.nA if net == N.NET_POP else env.p.nb * env.p.tax_levels
        out = {"value": torch.empty(rows, dtype=torch.float32, device=dev)}
        if sample:
            out["act"] = torch.empty((rows, heads), dtype=torch.int32, device=dev)
            out["logp"] = torch.empty(rows, dtype=torch.float32, device=dev)
        if entropy:
            out["entropy"] = torch.empty(rows, dtype=torch.float32, device=dev)
        if logits:
            out["logits"] = torch.empty((rows, O), dtype=torch.float32, device=dev)
        w = self.pop_w if net == N.NET_POP else self.gov_w
        rest = (_ptr(obs.contiguous()), _ptr(None if mask is None else mask.contiguous()),
                _ptr(None if u is None else u.contiguous()), _ptr(out.get("act")), _ptr(out.get("logp")),
                _ptr(out["value"]), _ptr(out.get("entropy")), _ptr(out.get("logits")), _stream(stream))
        if net == N.NET_POP and self.layout != N.NETS_SHARED:
            N.check(N.load().policy_forward_agents(C.byref(env.p), _ptr(env.state), self.layout, self.hidden,
                                                   self.precision, _ptr(w), *rest), "policy_forward_agents")
        else:
            N.check(N.load().policy_forward(C.byref(env.p), _ptr(env.state), net, self.hidden, self.precision,
                                            _ptr(w), *rest), "policy_forward")
        return out


class Rollout:
    """Buffers of a T-step rollout and the call that fills them."""

    def __init__(self, env: VecEnv, policy: Policy, T: int):
        self.env, self.policy, self.T = env, policy, T
        E, A, dev = env.E, env.A, env.device
        nb = env.p.nb
        f32, i32 = torch.float32, torch.int32
        self.buf = dict(
            obs=torch.empty((T + 1, E, A, env.D), dtype=f32, device=dev),
            gobs=torch.empty((T + 1, E, env.G), dtype=f32, device=dev),
            mask=torch.empty((T + 1, E, A, env.W), dtype=i32, device=dev),
            act=torch.empty((T, E, A), dtype=i32, device=dev),
            gact=torch.empty((T, E, nb), dtype=i32, device=dev),
            logp=torch.empty((T, E, A), dtype=f32, device=dev),
            glogp=torch.empty((T, E), dtype=f32, device=dev),
            value=torch.empty((T + 1, E, A), dtype=f32, device=dev),
            gvalue=torch.empty((T + 1, E), dtype=f32, device=dev),
            rew=torch.empty((T, E, A), dtype=f32, device=dev),
            grew=torch.empty((T, E), dtype=f32, device=dev),
            done=torch.empty((T, E), dtype=torch.uint8, device=dev),
        )
        self._c = N.EjRollout(**{k: v.data_ptr() for k, v in self.buf.items()})
        self.chains = None

    def reset(self, seed=0, pop_sizes=None):
        b = self.buf
        self.env.reset(seed=seed, pop_sizes=pop_sizes, out=dict(obs=b["obs"][0], gobs=b["gobs"][0], mask=b["mask"][0]))

    def carry_over(self):
        """Start the next rollout from the last observation."""
        for k in ("obs", "gobs", "mask"):
            self.buf[k][0].copy_(self.buf[k][self.T])

    def capture(self):
        """Capture carry_over + run (the slot-0 copies and 2T + 1 launches per
        chain in BF16, 3T + 2 in FP32) as one CUDA graph; replay() then runs
        the next rollout.  Runs one rollout eagerly first (kernel attributes
        and the chains' streams are set up outside the capture)."""
        self.carry_over()
        self.run()
        torch.cuda.synchronize(self.env.device)
        s = torch.cuda.Stream(device=self.env.device)
        s.wait_stream(torch.cuda.current_stream(self.env.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.carry_over()
                self.run(stream=s)
        torch.cuda.current_stream(self.env.device).wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        """The next rollout (carry_over + run) as one graph launch."""
        self.graph.replay()
        return self.buf

    def run(self, stream=None, chains=None):
        """One T-step rollout.  `chains` (1..4, default self.chains) splits
        the environments into independent chains on as many streams; None:
        the library's choice (2 chains from 2048 environments).  The result
        is the same for every choice."""
        pol = self.policy
        n = self.chains if chains is None else chains
        lib = N.load()
        if pol.layout != N.NETS_SHARED:
            N.check(lib.rollout_agents(C.byref(self.env.p), _ptr(self.env.state), self.T, pol.hidden, pol.precision,
                                       pol.layout, _ptr(pol.pop_w), _ptr(pol.gov_w), C.byref(self._c),
                                       _stream(stream)), "rollout_agents")
            return self.buf
        args = (C.byref(self.env.p), _ptr(self.env.state), self.T, pol.hidden, pol.precision, _ptr(pol.pop_w),
                _ptr(pol.gov_w), C.byref(self._c))
        if n is None:
            N.check(lib.rollout(*args, _stream(stream)), "rollout")
        else:
            N.check(lib.rollout_split(*args, int(n), _stream(stream)), "rollout_split")
        return self.buf
