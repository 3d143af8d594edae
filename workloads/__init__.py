"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the propagation method itself: it draws
random numbers (its own SplitMix64 stream, so that values do not depend on the
numpy version or the machine) and builds the model operators (Hamiltonian,
jump operators, drive operator) and the random density matrices that the
method consumes.  Neither the oracle nor the CUDA path is imported here.
"""

from .rng import splitmix64, uniform01, normal, ginibre_states, stream_seed
from .transmon import (
    annihilation,
    transmon_chain,
    paper_grape_model,
    TransmonModel,
)
from .configs import CONFIGS, make_workload

__all__ = [
    "splitmix64",
    "uniform01",
    "normal",
    "ginibre_states",
    "stream_seed",
    "annihilation",
    "transmon_chain",
    "paper_grape_model",
    "TransmonModel",
    "CONFIGS",
    "make_workload",
]
