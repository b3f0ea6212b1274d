"""Rollouts over environments of uneven population and action-space sizes.

Environments differ in population A_e and in the number of price levels P_e
(P_e in {5, 10, 20}: prices (k + 1) * 10 / P, so 24, 44 or 84 actions at two
resources).  They are partitioned into classes; a class shares one state
buffer whose CTA size follows its largest population (agents above an
environment's own population are inactive), one population network per
action-space size (weights shared by all classes with that P) and the
government network.  Each class runs the library's rollout (policy,
government policy and env_step per step) on its own stream; the T-step
rollouts of all classes are captured as parallel branches of one CUDA graph,
so a whole batched rollout is one graph launch.

The partition is a tuning choice: ``exact`` (one class per distinct
(P, population)), ``pow2`` (populations rounded up to a power of two: one CTA
size per class), ``coarse`` (populations up to 64, up to 256, larger) or
``by_actions`` (one class per P, CTA size of the largest population).  ``autotune`` times a short captured rollout of each and keeps
the fastest.
"""
from __future__ import annotations

import time
from collections import OrderedDict

import torch

from .env import VecEnv
from .policy import Policy, Rollout


def price_grid(P: int):
    """Price levels (k + 1) * 10 / P, k < P, as a tick and integer multiples."""
    return dict(P=P, price_tick=10.0 / P, price_ticks=list(range(1, P + 1)))


def _pow2(a):
    n = 32
    while n < a:
        n *= 2
    return n


def plan_classes(pops, levels, granularity):
    """[(P, A_max, env indices)] for a partition granularity."""
    groups = OrderedDict()
    for e, (a, P) in enumerate(zip(pops, levels)):
        if granularity == "exact":
            key = (P, a)
        elif granularity == "pow2":
            key = (P, _pow2(a))
        elif granularity == "coarse":
            key = (P, 64 if a <= 64 else 256 if a <= 256 else 1024)
        elif granularity == "by_actions":
            key = (P,)
        else:
            raise ValueError(granularity)
        groups.setdefault(key, []).append(e)
    return [(key[0], max(pops[e] for e in idx), idx) for key, idx in sorted(groups.items())]


class BatchedRollout:
    def __init__(self, pops, levels, T, weights, hidden=128, precision="bf16", granularity="pow2",
                 device="cuda", **env_kw):
        """weights: {("pop", P): tensor, ("gov",): tensor} in the library's layout."""
        self.pops, self.levels, self.T = list(pops), list(levels), T
        self.device = torch.device(device)
        self.granularity = granularity
        self.classes = []
        for P, A_max, idx in plan_classes(self.pops, self.levels, granularity):
            env = VecEnv(len(idx), A_max, device=self.device, **price_grid(P), **env_kw)
            pol = Policy(env, weights[("pop", P)], weights[("gov",)], hidden=hidden, precision=precision)
            ro = Rollout(env, pol, T)
            pop = torch.tensor([self.pops[e] for e in idx], dtype=torch.int32, device=self.device)
            self.classes.append(dict(P=P, A_max=A_max, idx=idx, env=env, policy=pol, ro=ro, pop=pop,
                                     stream=torch.cuda.Stream(device=self.device)))
        self.graph = None

    @property
    def agent_steps(self):
        return sum(self.pops) * self.T

    def reset(self, seed=0):
        for k, c in enumerate(self.classes):
            c["ro"].reset(seed=seed + 7919 * k, pop_sizes=c["pop"])
        torch.cuda.synchronize(self.device)

    def _issue(self):
        """Every class's T-step rollout on its own stream, then the copy of its
        last observation into slot 0 for the next rollout."""
        main = torch.cuda.current_stream(self.device)
        for c in self.classes:
            c["stream"].wait_stream(main)
            with torch.cuda.stream(c["stream"]):
                c["ro"].run()
                c["ro"].carry_over()
        for c in self.classes:
            main.wait_stream(c["stream"])

    def capture(self):
        """Run once eagerly (sets kernel attributes), then capture one graph."""
        self._issue()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._issue()
        self.graph = g
        return g

    def run(self):
        if self.graph is None:
            self._issue()
        else:
            self.graph.replay()



def autotune(pops, levels, weights, T_probe=8, hidden=128, precision="bf16", candidates=None,
             device="cuda", repeats=3, **env_kw):
    """Times a captured T_probe-step batched rollout per partition; returns
    (best granularity, {granularity: agent-steps/s})."""
    candidates = candidates or ("exact", "pow2", "coarse", "by_actions")
    rates = {}
    for gran in candidates:
        br = BatchedRollout(pops, levels, T_probe, weights, hidden=hidden, precision=precision,
                            granularity=gran, device=device, **env_kw)
        br.reset(seed=1)
        br.capture()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for _ in range(repeats):
            br.run()
        torch.cuda.synchronize(device)
        rates[gran] = br.agent_steps * repeats / (time.perf_counter() - t0)
        del br
        torch.cuda.empty_cache()
    best = max(rates, key=rates.get)
    return best, rates
