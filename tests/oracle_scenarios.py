"""Helpers that drive the CPU oracle through hand-written scenarios.

Action ids follow the layout of the environment (NO-OP, gather per resource,
craft, buy per resource and price level, sell per resource and price level).
"""
from __future__ import annotations

import numpy as np

from oracle.env import OracleEnv, default_params

NOOP = 0


def gather(r):
    return 1 + r


def craft(R=2):
    return R + 1


def buy(r, level, R=2, P=5):
    return R + 2 + r * P + level


def sell(r, level, R=2, P=5):
    return R + 2 + R * P + r * P + level


class Scenario:
    """A tiny environment whose every input is chosen by the test."""

    def __init__(self, A, sg=None, sc=None, **params):
        self.p = default_params(**params)
        self.env = OracleEnv(self.p, A)
        self.A = A
        R = self.p["R"]
        sg = np.full((A, R), 1.0, np.float32) if sg is None else np.asarray(sg, np.float32)
        sc = np.full(A, 0.5, np.float32) if sc is None else np.asarray(sc, np.float32)
        self.sg, self.sc = sg, sc
        self.env.reset(sg, sc)
        self.last = None

    def step(self, acts, gov=(0, 0, 0), u=None, tb=None):
        A = self.A
        acts = np.asarray(acts, np.int32)
        u = np.zeros(A, np.float32) if u is None else np.asarray(u, np.float32)
        tb = np.arange(A, dtype=np.uint32) if tb is None else np.asarray(tb, np.uint32)
        self.last = self.env.step(acts, np.asarray(gov, np.int32), u, tb, self.sg, self.sc)
        return self.last

    def agents(self):
        return self.env.agents()
