"""Simultaneous PPO training of the population and government networks
(Section 4), driving the library's rollout and update calls.

Every step of the method runs in the library (rollout: policy forward,
sampling and env_step; update: GAE, minibatch gradients, Adam).  This module
only schedules the calls, anneals the learning rate and the entropy
coefficient as Table 2 states (learning rate linearly to 0 over the whole
run, entropy coefficient linearly to 0 over its first 90 %), and keeps
per-episode measurements on the host from the rollout buffers:

* population return: each agent's reward summed over an episode (Eq. 2 sums
  to the change of Eq. 1's utility), mean and median over the agents;
* social welfare at the episode's end (Eq. 3-5): its value at the start
  (every agent holds the starting coin, gini 0) plus the government rewards
  of the episode;
* productivity: total coin (escrow included) of the state one step before
  the end (the observation of the last state is the next episode's first,
  as environments restart in the same step), and equality = welfare /
  productivity;
* the tax rates the government sets at period starts.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _native as N
from .policy import Policy, Rollout
from .ppo import PPO


class EpisodeLog:
    """Per-environment sums over the running episode and the finished episodes."""

    def __init__(self, E: int, A: int, start_coin: float, T_tax: int):
        self.E, self.A, self.T_tax = E, A, T_tax
        self.welfare0 = start_coin * A
        self.ret = np.zeros((E, A))
        self.gsum = np.zeros(E)
        self.t = 0
        self.episodes = []           # dicts per finished episode
        self.rates = []              # (iteration, rates [E][nb]) at period starts

    def add(self, it: int, buf: dict):
        rew = buf["rew"].double().cpu().numpy()
        grew = buf["grew"].double().cpu().numpy()
        done = buf["done"].cpu().numpy()
        gobs = buf["gobs"][:, :, 0].double().cpu().numpy()
        gact = buf["gact"].cpu().numpy()
        T = rew.shape[0]
        for s in range(T):
            if self.t % self.T_tax == 0:
                self.rates.append((it, gact[s]))
            self.ret += rew[s]
            self.gsum += grew[s]
            self.t += 1
            ended = np.nonzero(done[s])[0]
            for e in ended:
                prod = float(gobs[s, e]) * self.A      # state after the episode's second-to-last step
                welfare = self.welfare0 + float(self.gsum[e])
                self.episodes.append(dict(iteration=it, mean_return=float(self.ret[e].mean()),
                                          median_return=float(np.median(self.ret[e])), welfare=welfare,
                                          productivity=prod, equality=welfare / prod if prod > 0 else 0.0))
            if len(ended):
                self.ret[ended] = 0.0
                self.gsum[ended] = 0.0
                self.t = 0 if done[s].all() else self.t


class Trainer:
    """PPO on a Policy's networks with Table 2's schedule."""

    def __init__(self, policy: Policy, T: int = 150, precision: str = "bf16", total_iterations: int = 100,
                 lr: float = 5e-4, ent_coef: float = 0.1, seed: int = 0, **ppo_params):
        self.policy, self.env, self.T = policy, policy.env, T
        self.rollout = Rollout(self.env, policy, T)
        self.ppo = PPO(policy, T, precision=precision, seed=seed, **ppo_params)
        self.lr0, self.ent0 = lr, ent_coef
        self.total = max(1, int(total_iterations))
        self.it = 0
        p = self.env.params
        self.log = EpisodeLog(self.env.E, self.env.A, p["start_coin"], p["T_tax"])

    def reset(self, seed: int = 0):
        self.rollout.reset(seed=seed)

    def iteration(self):
        """One rollout of T steps and one PPO update (both networks)."""
        frac = self.it / self.total
        self.ppo.pp.lr = self.lr0 * (1.0 - frac)
        self.ppo.pp.ent_coef = self.ent0 * max(0.0, 1.0 - frac / 0.9)
        if self.it:
            self.rollout.carry_over()
        self.rollout.run()
        self.log.add(self.it, self.rollout.buf)
        stats = self.ppo.update(self.rollout)
        self.it += 1
        return stats

    def train(self, iterations: int | None = None):
        n = self.total - self.it if iterations is None else iterations
        t0 = time.perf_counter()
        for _ in range(n):
            self.iteration()
        torch.cuda.synchronize(self.env.device)
        return time.perf_counter() - t0

    def summary(self, window: float = 0.1):
        """Episode measurements averaged over the first and the last `window`
        of the finished episodes, and the mean tax rates of the last window
        of period starts."""
        ep = self.log.episodes
        if not ep:
            return {}
        k = max(1, int(len(ep) * window))
        keys = ("mean_return", "median_return", "welfare", "productivity", "equality")
        first = {f: float(np.mean([e[f] for e in ep[:k]])) for f in keys}
        last = {f: float(np.mean([e[f] for e in ep[-k:]])) for f in keys}
        out = {"episodes": len(ep), "first": first, "last": last, "episodes_per_window": k}
        if self.log.rates and self.env.params["gov_enabled"]:
            kr = max(1, int(len(self.log.rates) * window))
            lev = np.stack([r for _, r in self.log.rates[-kr:]]).reshape(-1, self.env.p.nb)
            out["last_tax_rates"] = (lev.mean(axis=0) / (self.env.p.tax_levels - 1)).tolist()
        return out
