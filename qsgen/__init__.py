"""Seeded input generators shared by the oracle and the CUDA path (no simulation arithmetic)."""

from .rng import SplitMix64  # noqa: F401
from .circuits import *  # noqa: F401,F403
