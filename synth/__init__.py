"""Seeded synthetic inputs for the EconoJax hot path.

This package holds no arithmetic of the simulated economy.  It turns a seed
into the random draws the method consumes (uniform random actions, gather
draws, tie-break keys, government rate levels, skills, policy-sampling
uniforms) through Philox-4x32-10, with the counter mapping that
``include/econojax.h`` documents.  It is the one piece that both the CPU
oracle (through the tests) and the CUDA library's users share.
"""
from .philox import philox4x32_10, seed_key, u01, below  # noqa: F401
from .draws import (  # noqa: F401
    STREAM_POP, STREAM_GOV, STREAM_SKILL,
    pop_draws, gov_draws, skill_draws, episode_inputs,
)
from .weights import STREAM_WEIGHTS, net_layout, net_offsets, net_weights, pack, unpack  # noqa: F401
