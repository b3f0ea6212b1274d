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

With ``merge`` the policy launches of a step are merged across classes:
the population networks (one per price grid) and the government network of
all classes run as one launch of the BF16 kernel, which splits its CTAs
between the networks by rows (policy_forward_segments, one table entry per
class and network); then each class's env_step runs on its own stream.  Per
step the graph holds one policy node and one env_step node per class instead
of three launches per class.  The values, actions and states are those of the
per-class rollouts, bit for bit.  With ``chains`` N as well, every class is
split into N parts and part k of every class forms chain k: each chain's
merged policy launch and env_steps run on a stream of its own, the chains
interleaved step by step, so one chain's env_steps run beside another
chain's policy launch.

The partition is a tuning choice: ``exact`` (one class per distinct
(P, population)), ``pow2`` (populations rounded up to a power of two: one CTA
size per class), ``coarse`` (populations up to 64, up to 256, larger) or
``by_actions`` (one class per P, CTA size of the largest population).  ``autotune`` times a short captured rollout of each and keeps
the fastest.
"""
from __future__ import annotations

import time
from collections import OrderedDict

import ctypes as C

import torch

from . import _native as N
from .env import VecEnv, _ptr, _stream
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
                 device="cuda", merge=False, chains=None, **env_kw):
        """weights: {("pop", P): tensor, ("gov",): tensor} in the library's layout.
        chains: independent chains of environments (1..4; None: the library's
        choice): per class rollout for the unmerged rollouts; with merge,
        every class is split into that many contiguous parts, part k of every
        class forming chain k, whose merged policy launches and env_steps run
        on a stream of their own (one chain's env_steps beside another's
        policy launch)."""
        self.pops, self.levels, self.T = list(pops), list(levels), T
        self.device = torch.device(device)
        self.granularity = granularity
        self.merge = merge
        self.chains = chains
        # one device copy per network: classes with the same price grid share it
        weights = {k: v.to(self.device, torch.float32).contiguous() for k, v in weights.items()}
        self.classes = []
        n_split = int(chains) if (merge and chains) else 1
        for ci, (P, A_max, idx) in enumerate(plan_classes(self.pops, self.levels, granularity)):
            for q in range(n_split):
                part = idx[len(idx) * q // n_split: len(idx) * (q + 1) // n_split]
                if not part:
                    continue
                k = (q + ci) % n_split           # rotated per class: small classes spread over the chains
                env = VecEnv(len(part), A_max, device=self.device, **price_grid(P), **env_kw)
                pol = Policy(env, weights[("pop", P)], weights[("gov",)], hidden=hidden, precision=precision)
                ro = Rollout(env, pol, T)
                ro.chains = None if (chains is None or merge) else max(1, min(int(chains), len(part)))
                pop = torch.tensor([self.pops[e] for e in part], dtype=torch.int32, device=self.device)
                self.classes.append(dict(P=P, A_max=A_max, idx=part, env=env, policy=pol, ro=ro, pop=pop, chain=k,
                                         stream=torch.cuda.Stream(device=self.device)))
        # one stream per merged chain beyond the first (the first runs on the caller's stream)
        self.chain_ids = sorted({c["chain"] for c in self.classes})
        self.chain_streams = {k: torch.cuda.Stream(device=self.device) for k in self.chain_ids[1:]}
        self.graph = None

    @property
    def agent_steps(self):
        return sum(self.pops) * self.T

    def reset(self, seed=0):
        for k, c in enumerate(self.classes):
            c["ro"].reset(seed=seed + 7919 * k, pop_sizes=c["pop"])
        torch.cuda.synchronize(self.device)

    def _policies(self, t, stream, classes=None):
        """Step t's policy launches of the given classes (default: all;
        population and government networks) in one policy_forward_segments
        call (t = T: values only)."""
        classes = self.classes if classes is None else classes
        n = 2 * len(classes)
        last = t == self.T
        V = C.c_void_p * n
        segs = [(c, net) for c in classes for net in (N.NET_POP, N.NET_GOV)]

        def buf(c, pop_key, gov_key, net):
            return _ptr(c["ro"].buf[pop_key if net == N.NET_POP else gov_key][t])

        pol = self.classes[0]["policy"]
        N.check(N.load().policy_forward_segments(
            n, V(*[C.addressof(c["env"].p) for c, _ in segs]), V(*[_ptr(c["env"].state) for c, _ in segs]),
            (C.c_int32 * n)(*[net for _, net in segs]),
            V(*[_ptr(c["policy"].pop_w if net == N.NET_POP else c["policy"].gov_w) for c, net in segs]),
            pol.hidden, pol.precision, V(*[buf(c, "obs", "gobs", net) for c, net in segs]),
            V(*[buf(c, "mask", None, net) if net == N.NET_POP else None for c, net in segs]),
            None if last else V(*[buf(c, "act", "gact", net) for c, net in segs]),
            None if last else V(*[buf(c, "logp", "glogp", net) for c, net in segs]),
            V(*[buf(c, "value", "gvalue", net) for c, net in segs]), _stream(stream)),
            "policy_forward_segments")

    def _issue_merged(self):
        """T + 1 steps of {a chain's classes' policies in one call on the
        chain's stream, then each of its classes' env_step on its own
        stream}, chains interleaved step by step, then the slot-0 copies."""
        main = torch.cuda.current_stream(self.device)
        T = self.T
        cs = {k: (main if k == self.chain_ids[0] else self.chain_streams[k]) for k in self.chain_ids}
        members = {k: [c for c in self.classes if c["chain"] == k] for k in self.chain_ids}
        for k in self.chain_ids[1:]:
            cs[k].wait_stream(main)
        for t in range(T + 1):
            for k in self.chain_ids:
                self._policies(t, cs[k], members[k])
                if t == T:
                    continue
                for c in members[k]:
                    c["stream"].wait_stream(cs[k])
                    b = c["ro"].buf
                    c["env"].step(1, act=b["act"][t], gov_act=b["gact"][t], stream=c["stream"],
                                  out=dict(rew=b["rew"][t:t + 1], grew=b["grew"][t:t + 1],
                                           done=b["done"][t:t + 1], obs=b["obs"][t + 1:t + 2],
                                           gobs=b["gobs"][t + 1:t + 2], mask=b["mask"][t + 1:t + 2]))
                for c in members[k]:
                    cs[k].wait_stream(c["stream"])
        for k in self.chain_ids[1:]:
            main.wait_stream(cs[k])
        for c in self.classes:
            c["ro"].carry_over()

    def _issue(self):
        """Every class's T-step rollout on its own stream, then the copy of its
        last observation into slot 0 for the next rollout."""
        if self.merge:
            return self._issue_merged()
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



def parse_candidate(cand: str):
    """"gran[+merge][+chainsN]" -> (granularity, merge, chains)."""
    parts = cand.split("+")
    gran, merge, chains = parts[0], False, None
    plan_classes([1], [5], gran)                       # validates the granularity
    for p in parts[1:]:
        if p == "merge":
            merge = True
        elif p.startswith("chains") and p[6:].isdigit() and 1 <= int(p[6:]) <= 4:
            chains = int(p[6:])
        else:
            raise ValueError(cand)
    return gran, merge, chains


def autotune(pops, levels, weights, T_probe=64, hidden=128, precision="bf16", candidates=None,
             device="cuda", repeats=5, **env_kw):
    """Times a captured T_probe-step batched rollout per candidate (CUDA
    events on the replaying stream, the median of `repeats` replays; the probe
    must be long enough that a replay's fixed costs, such as the per-class
    copies of the last observation, do not decide between candidates with
    different class counts); returns
    (best candidate, {candidate: agent-steps/s}).  A candidate is a partition
    granularity (the environment CTA size of each class follows from it),
    with "+merge" for merged policy launches ("exact+merge") and "+chainsN"
    for N independent chains of environments (per class rollout, or with
    "+merge" each class split into N parts forming N merged chains), so that
    policy launches and env_steps of different chains overlap."""
    candidates = candidates or ("exact", "pow2", "coarse", "by_actions", "exact+merge", "coarse+merge",
                                "exact+merge+chains2", "exact+chains1", "exact+chains2", "pow2+chains2")
    rates = {}
    parsed = {cand: parse_candidate(cand) for cand in candidates}    # every name checked before any work
    for cand in candidates:
        gran, merged, chains = parsed[cand]
        br = BatchedRollout(pops, levels, T_probe, weights, hidden=hidden, precision=precision,
                            granularity=gran, merge=merged, chains=chains, device=device, **env_kw)
        br.reset(seed=1)
        br.capture()
        br.run()
        torch.cuda.synchronize(device)
        ms = []
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            br.run()
            b.record()
            torch.cuda.synchronize(device)
            ms.append(a.elapsed_time(b))
        ms.sort()
        rates[cand] = br.agent_steps / (ms[len(ms) // 2] / 1e3)
        del br
        torch.cuda.empty_cache()
    best = max(rates, key=rates.get)
    return best, rates
