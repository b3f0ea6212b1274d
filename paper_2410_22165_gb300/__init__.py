"""GB300-native (sm_103a) EconoJax hot path (arxiv 2410.22165).

``VecEnv`` runs E environments of population agents and a government on the
GPU through the C ABI of ``include/econojax.h`` (library: libeconojax.so,
built by ``paper_2410_22165_gb300.build``).
"""
from ._native import EjError, load  # noqa: F401
from .env import VecEnv  # noqa: F401
from .policy import Policy, Rollout  # noqa: F401
from .ppo import PPO, PPOLoss  # noqa: F401
from .batch import BatchedRollout, autotune, plan_classes, price_grid  # noqa: F401
