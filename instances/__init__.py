"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle's tests.

This package generates problem *data* only: Exact-Cover-3 clause lists (with their unique
solution), random qubit pairs with couplings, and random state vectors.  It contains none of
the method's arithmetic (no Hamiltonian construction, no matvec, no integrator): each side
builds its own Hamiltonian from these data.
"""
from .rng import SplitMix64
from .ec3 import EC3Instance, generate_ec3, generate_ec3_hard, count_solutions, xx_pairs
from .vectors import random_state, uniform_state_value

__all__ = [
    "SplitMix64",
    "EC3Instance",
    "generate_ec3",
    "generate_ec3_hard",
    "count_solutions",
    "xx_pairs",
    "random_state",
    "uniform_state_value",
]
